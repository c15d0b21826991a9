"""Python binding of libgbs: argument marshalling between torch/numpy and the C ABI.

Every step of the computation runs in libgbs's CUDA kernels; torch provides
device memory and the stream only.  Names follow include/gbs.h.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import GbsError, GBS_FP64, GBS_FP32_SPLIT, GBS_DD, GBS_FX, GBS_FF, GBS_AUTO, GBS_FX192

PRECISIONS = {"fp64": GBS_FP64, "fp32": GBS_FP32_SPLIT, "dd": GBS_DD, "fx": GBS_FX, "ff": GBS_FF,
              "auto": GBS_AUTO, "fx192": GBS_FX192, GBS_FP64: GBS_FP64, GBS_FP32_SPLIT: GBS_FP32_SPLIT,
              GBS_DD: GBS_DD, GBS_FX: GBS_FX, GBS_FF: GBS_FF, GBS_AUTO: GBS_AUTO, GBS_FX192: GBS_FX192}


def _ptr(t) -> ctypes.c_void_p:
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _dev_f64(x, device) -> torch.Tensor:
    if isinstance(x, torch.Tensor):
        return x.to(device=device, dtype=torch.float64).contiguous()
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device=device)


def _complex_interleaved(U, device) -> torch.Tensor:
    if isinstance(U, torch.Tensor):
        U = U.to(device=device, dtype=torch.complex128).contiguous()
        return torch.view_as_real(U).contiguous()
    U = np.ascontiguousarray(U, dtype=np.complex128)
    return torch.as_tensor(U.view(np.float64).reshape(U.shape[0], -1), device=device)


def patterns_tensor(patterns, device) -> torch.Tensor:
    """(n, 2) int64 tensor holding the uint64 pattern words bit for bit."""
    if isinstance(patterns, torch.Tensor):
        return patterns.to(device=device, dtype=torch.int64).contiguous()
    a = np.ascontiguousarray(patterns, dtype=np.uint64).reshape(-1, 2)
    return torch.as_tensor(a.view(np.int64), device=device)


class Context:
    """A libgbs context bound to one CUDA device and one stream."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        self.lib = _lib.load()
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        code = self.lib.gbs_create(ctypes.byref(h), device, ctypes.c_void_p(self.stream.cuda_stream))
        if code:
            raise GbsError(code, "gbs_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.gbs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, code: int):
        if code:
            raise GbsError(code, self.lib.gbs_last_error(self.h).decode())

    def set_stream(self, stream: torch.cuda.Stream):
        self.stream = stream
        self._check(self.lib.gbs_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream)))

    def reserve(self, n_pat: int, n_max: int):
        self._check(self.lib.gbs_reserve(self.h, n_pat, n_max))

    def click_distribution(self, O: torch.Tensor, logdet: torch.Tensor):
        """(log p(n), kappa_n) for n = 0..M: the whole device's click-number distribution."""
        M = O.shape[0] // 2
        logp = torch.empty(M + 1, dtype=torch.float64, device=self.device)
        kappa = torch.empty(M + 1, dtype=torch.float64, device=self.device)
        self._check(self.lib.gbs_click_distribution(self.h, M, _ptr(O), _ptr(logdet), _ptr(logp), _ptr(kappa)))
        return logp, kappa

    def sector_distribution(self, O: torch.Tensor, logdet: torch.Tensor, L: int = 256, rho: float = 1.0,
                            K: int | None = None, even_only: bool = False, precision="fp64"):
        """p_k(n) for k = 0..K, n = 0..M ((K + 1) x (M + 1), device): the photon-number
        sectors of the whole device's click-number distribution, from L circle points
        (even_only: the state is lossless, odd sectors vanish; half the sweeps)."""
        M = O.shape[0] // 2
        K = L - 1 if K is None else K
        pkn = torch.empty((K + 1, M + 1), dtype=torch.float64, device=self.device)
        self._check(self.lib.gbs_sector_distribution(self.h, M, _ptr(O), _ptr(logdet), int(L), float(rho), int(K),
                                                     int(bool(even_only)), PRECISIONS[precision], _ptr(pkn)))
        return pkn

    def approx_sector_curves(self, O: torch.Tensor, logdet: torch.Tensor, pattern, order: int = 4,
                             precision="ff", K: int = 255):
        """The order-j fit of every photon-number sector of one pattern S with n clicks:
        (K + 1) x (n + 1) device tensor, row k = the estimate of P(c clicks in S, k photons)
        at column c; plus the pattern's (logP, status)."""
        M = O.shape[0] // 2
        pats = patterns_tensor(pattern, self.device)[:1]
        pat = pats.cpu().numpy()[0]
        n = sum(bin(int(w) & 0xFFFFFFFFFFFFFFFF).count("1") for w in pat)
        curves = torch.empty((K + 1, n + 1), dtype=torch.float64, device=self.device)
        logP = torch.empty(1, dtype=torch.float64, device=self.device)
        status = torch.empty(1, dtype=torch.int32, device=self.device)
        self._check(self.lib.gbs_approx_sector_curves(self.h, M, _ptr(O), _ptr(logdet), _ptr(pats), n, int(order),
                                                      PRECISIONS[precision], int(K), _ptr(curves), _ptr(logP),
                                                      _ptr(status)))
        return curves, logP, status

    def autotune(self, O: torch.Tensor, logdet: torch.Tensor, patterns, precision="fx"):
        """Pick the exact sweep's work split for this precision on these patterns
        (kept in the context); returns (split, ms of one sweep).  Synchronous; call it
        before reserve()."""
        M = O.shape[0] // 2
        pats = patterns_tensor(patterns, self.device)
        s, ms = ctypes.c_int(), ctypes.c_double()
        self._check(self.lib.gbs_autotune(self.h, M, _ptr(O), _ptr(logdet), _ptr(pats), pats.shape[0],
                                          PRECISIONS[precision], ctypes.byref(s), ctypes.byref(ms)))
        return s.value, ms.value

    def build_state(self, U, r, eta: float, want_sigma: bool = False, check: bool = True):
        """Device O (2M x 2M), log det sigma_Q (1,), sigma (or None), status (1,) int32."""
        Ud = _complex_interleaved(U, self.device)
        M = Ud.shape[0]
        rd = _dev_f64(r, self.device)
        O = torch.empty((2 * M, 2 * M), dtype=torch.float64, device=self.device)
        logdet = torch.empty(1, dtype=torch.float64, device=self.device)
        sigma = torch.empty_like(O) if want_sigma else None
        status = None if check else torch.zeros(1, dtype=torch.int32, device=self.device)
        self._check(self.lib.gbs_build_state(self.h, M, _ptr(Ud), _ptr(rd), float(eta), _ptr(sigma),
                                             _ptr(O), _ptr(logdet), _ptr(status)))
        return dict(O=O, logdet=logdet, sigma=sigma, status=status)

    def prob(self, O: torch.Tensor, logdet: torch.Tensor, patterns, order: int = 0,
             precision="auto", out=None):
        """log P per pattern (device tensors): dict(logP, kappa, err_bound, status).
        precision "auto": the exact sum in 128-bit fixed point with a double-double rerun of
        the patterns outside its range; the approximation with float-float minors."""
        M = O.shape[0] // 2
        pats = patterns_tensor(patterns, self.device)
        n_pat = pats.shape[0]
        if out is None:
            out = dict(logP=torch.empty(n_pat, dtype=torch.float64, device=self.device),
                       kappa=torch.empty(n_pat, dtype=torch.float64, device=self.device),
                       err_bound=torch.empty(n_pat, dtype=torch.float64, device=self.device),
                       status=torch.empty(n_pat, dtype=torch.int32, device=self.device))
        self._check(self.lib.gbs_prob(self.h, M, _ptr(O), _ptr(logdet), _ptr(pats), n_pat, order,
                                      PRECISIONS[precision], _ptr(out["logP"]), _ptr(out["kappa"]),
                                      _ptr(out["err_bound"]), _ptr(out["status"])))
        return out

    def prob_noalloc(self, O: torch.Tensor, logdet: torch.Tensor, patterns, n_max: int,
                     precision="fp64", out=None):
        """Exact log P without any device allocation inside the library (its scratch is a
        fixed array in the library's device memory); out buffers are the caller's."""
        M = O.shape[0] // 2
        pats = patterns_tensor(patterns, self.device)
        n_pat = pats.shape[0]
        if out is None:
            out = dict(logP=torch.empty(n_pat, dtype=torch.float64, device=self.device),
                       kappa=torch.empty(n_pat, dtype=torch.float64, device=self.device),
                       err_bound=torch.empty(n_pat, dtype=torch.float64, device=self.device),
                       status=torch.empty(n_pat, dtype=torch.int32, device=self.device))
        self._check(self.lib.gbs_prob_noalloc(self.h, M, _ptr(O), _ptr(logdet), _ptr(pats), n_pat, n_max,
                                              PRECISIONS[precision], _ptr(out["logP"]), _ptr(out["kappa"]),
                                              _ptr(out["err_bound"]), _ptr(out["status"])))
        return out

    def prob_partial(self, O: torch.Tensor, patterns, part: int, nparts: int, precision="fx"):
        """Slice `part` of `nparts` of the batch's exact-sum work units: per pattern the
        slice's partial sum (T_hi, T_lo, sum |terms|) as an (n_pat, 3) tensor and its flags
        (n_pat int32)."""
        M = O.shape[0] // 2
        pats = patterns_tensor(patterns, self.device)
        n_pat = pats.shape[0]
        partial = torch.empty((n_pat, 3), dtype=torch.float64, device=self.device)
        pflag = torch.empty(n_pat, dtype=torch.int32, device=self.device)
        self._check(self.lib.gbs_prob_partial(self.h, M, _ptr(O), _ptr(pats), n_pat, PRECISIONS[precision],
                                              part, nparts, _ptr(partial), _ptr(pflag)))
        return partial, pflag

    def prob_combine(self, logdet: torch.Tensor, patterns, partials: torch.Tensor, pflags: torch.Tensor,
                     precision="fx"):
        """The slices' partial sums (nparts, n_pat, 3) and flags (nparts, n_pat), in part
        order, combined into what prob() returns for the batch."""
        pats = patterns_tensor(patterns, self.device)
        n_pat = pats.shape[0]
        parts = partials.to(device=self.device, dtype=torch.float64).contiguous()
        flags = pflags.to(device=self.device, dtype=torch.int32).contiguous()
        out = dict(logP=torch.empty(n_pat, dtype=torch.float64, device=self.device),
                   kappa=torch.empty(n_pat, dtype=torch.float64, device=self.device),
                   err_bound=torch.empty(n_pat, dtype=torch.float64, device=self.device),
                   status=torch.empty(n_pat, dtype=torch.int32, device=self.device))
        self._check(self.lib.gbs_prob_combine(self.h, _ptr(logdet), _ptr(pats), n_pat, PRECISIONS[precision],
                                              parts.shape[0], _ptr(parts), _ptr(flags), _ptr(out["logP"]),
                                              _ptr(out["kappa"]), _ptr(out["err_bound"]), _ptr(out["status"])))
        return out

    def run_host(self, U, r, eta: float, patterns, order: int = 0, precision="auto", out=None):
        """The whole path from host (numpy) buffers; returns numpy arrays."""
        U = np.ascontiguousarray(U, dtype=np.complex128)
        M = U.shape[0]
        r = np.ascontiguousarray(r, dtype=np.float64)
        pats = np.ascontiguousarray(patterns, dtype=np.uint64).reshape(-1, 2)
        n_pat = pats.shape[0]
        if out is None:
            out = dict(logP=np.empty(n_pat), kappa=np.empty(n_pat), err_bound=np.empty(n_pat),
                       status=np.empty(n_pat, dtype=np.int32))
        c = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        self._check(self.lib.gbs_run_host(self.h, M, c(U), c(r), float(eta), c(pats), n_pat, order,
                                          PRECISIONS[precision], c(out["logP"]), c(out["kappa"]),
                                          c(out["err_bound"]), c(out["status"])))
        return out

    def gen_patterns(self, seed: int, stream: int, M: int, n_lo: int, n_hi: int, n_pat: int):
        out = torch.empty((n_pat, 2), dtype=torch.int64, device=self.device)
        self._check(self.lib.gbs_gen_patterns(self.h, seed, stream, M, n_lo, n_hi, n_pat, _ptr(out)))
        return out

    def timing(self, enable: bool = True):
        self._check(self.lib.gbs_timing_enable(self.h, 1 if enable else 0))

    def timing_read(self, reset: bool = True):
        """(summed device ms, launches) of the sweep kernel since the last reset."""
        ms, n = ctypes.c_double(), ctypes.c_longlong()
        self._check(self.lib.gbs_timing_read(self.h, 1 if reset else 0, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def build_state_into(self, Ud: torch.Tensor, rd: torch.Tensor, eta: float, O: torch.Tensor,
                         logdet: torch.Tensor, status: torch.Tensor):
        """State build into preallocated device buffers (U interleaved (M, 2M) f64); no sync."""
        self._check(self.lib.gbs_build_state(self.h, Ud.shape[0], _ptr(Ud), _ptr(rd), float(eta), None,
                                             _ptr(O), _ptr(logdet), _ptr(status)))

    def grad(self, O: torch.Tensor, logdet: torch.Tensor, patterns, w: torch.Tensor):
        """dL/dsigma_Q for L = sum_p w_p log P_p; also the double-double log P and status."""
        M = O.shape[0] // 2
        pats = patterns_tensor(patterns, self.device)
        n_pat = pats.shape[0]
        w = w.to(device=self.device, dtype=torch.float64).contiguous()
        dsq = torch.empty_like(O)
        logP = torch.empty(n_pat, dtype=torch.float64, device=self.device)
        status = torch.empty(n_pat, dtype=torch.int32, device=self.device)
        self._check(self.lib.gbs_grad(self.h, M, _ptr(O), _ptr(logdet), _ptr(pats), n_pat, _ptr(w), _ptr(dsq),
                                      _ptr(logP), _ptr(status)))
        return dsq, logP, status

    def grad_approx(self, O: torch.Tensor, logdet: torch.Tensor, patterns, w: torch.Tensor, order: int = 4):
        """dL/dsigma_Q for L = sum_p w_p log P_p with the order-j approximation of every P_p
        (FP64 minors); also the forward's log P and status."""
        M = O.shape[0] // 2
        pats = patterns_tensor(patterns, self.device)
        n_pat = pats.shape[0]
        w = w.to(device=self.device, dtype=torch.float64).contiguous()
        dsq = torch.empty_like(O)
        logP = torch.empty(n_pat, dtype=torch.float64, device=self.device)
        status = torch.empty(n_pat, dtype=torch.int32, device=self.device)
        self._check(self.lib.gbs_grad_approx(self.h, M, _ptr(O), _ptr(logdet), _ptr(pats), n_pat, int(order),
                                             _ptr(w), _ptr(dsq), _ptr(logP), _ptr(status)))
        return dsq, logP, status

    def grad_params(self, Ud: torch.Tensor, rd: torch.Tensor, eta: float, dsq: torch.Tensor):
        """(dU interleaved (M, 2M), dr (M,), deta (1,)) from dL/dsigma_Q."""
        M = Ud.shape[0]
        dU = torch.empty_like(Ud)
        dr = torch.empty_like(rd)
        deta = torch.empty(1, dtype=torch.float64, device=self.device)
        self._check(self.lib.gbs_grad_params(self.h, M, _ptr(Ud), _ptr(rd), float(eta), _ptr(dsq), _ptr(dU),
                                             _ptr(dr), _ptr(deta)))
        return dU, dr, deta

    def clements_unitary(self, theta: torch.Tensor, phi: torch.Tensor, M: int) -> torch.Tensor:
        """U (M, 2M) interleaved complex from the mesh phases (device)."""
        U = torch.empty((M, 2 * M), dtype=torch.float64, device=self.device)
        th = theta.to(device=self.device, dtype=torch.float64).contiguous()
        ph = phi.to(device=self.device, dtype=torch.float64).contiguous()
        self._check(self.lib.gbs_clements_unitary(self.h, M, _ptr(th), _ptr(ph), _ptr(U)))
        return U

    def clements_grad(self, theta, phi, Ud, dU):
        th = theta.to(device=self.device, dtype=torch.float64).contiguous()
        ph = phi.to(device=self.device, dtype=torch.float64).contiguous()
        dth, dph = torch.empty_like(th), torch.empty_like(ph)
        self._check(self.lib.gbs_clements_grad(self.h, Ud.shape[0], _ptr(th), _ptr(ph), _ptr(Ud), _ptr(dU),
                                               _ptr(dth), _ptr(dph)))
        return dth, dph

    def set_pair_from(self, n_min: int = 80):
        """Approximation: patterns of at least n_min clicks take the CTA-pair minors kernel."""
        self._check(self.lib.gbs_set_pair_from(self.h, int(n_min)))

    def peak_flops(self, kind: str = "fp32") -> float:
        """FLOP/s of the FP32 / FP64 FMA loops ("fp32", "fp64") or of the fused
        Schur-update loops in double-double / fixed point ("dd", "fx"); "imad": 32-bit
        integer multiply-adds per second."""
        v = ctypes.c_double()
        code = {"fp32": 0, "fp64": 1, "dd": 2, "fx": 3, "imad": 4}[kind]
        self._check(self.lib.gbs_peak_flops(self.h, code, ctypes.byref(v)))
        return v.value


def grad_sharded(ctx, O: torch.Tensor, logdet: torch.Tensor, patterns, w, order: int = 0, group=None):
    """dL/dsigma_Q for L = sum_p w_p log P_p over a batch shared by the ranks of a
    torch.distributed process group (NCCL for CUDA tensors): rank k evaluates
    patterns k, k + N, k + 2N, ... (round robin, so that the pattern sizes, and with
    them the work, spread evenly) with ctx.grad (order 0) or ctx.grad_approx (order
    1..4), and one all-reduce (sum) of the 2M x 2M result combines the ranks: the
    gradient is linear in w, its -1/2 (sum w) A term included.  Without an
    initialised process group it is the one-rank case.  Returns (dL/dsigma_Q, this
    rank's pattern indices, their log P, their status)."""
    import torch.distributed as dist
    dist_on = dist.is_available() and dist.is_initialized()
    world = dist.get_world_size(group) if dist_on else 1
    rank = dist.get_rank(group) if dist_on else 0
    pats = patterns_tensor(patterns, O.device)
    wt = _dev_f64(w, O.device)
    idx = torch.arange(rank, pats.shape[0], world, device=O.device)
    if idx.numel():
        if order == 0:
            dsq, logP, status = ctx.grad(O, logdet, pats[idx], wt[idx])
        else:
            dsq, logP, status = ctx.grad_approx(O, logdet, pats[idx], wt[idx], order)
    else:
        dsq = torch.zeros_like(O)
        logP = torch.empty(0, dtype=torch.float64, device=O.device)
        status = torch.empty(0, dtype=torch.int32, device=O.device)
    if world > 1:
        dist.all_reduce(dsq, op=dist.ReduceOp.SUM, group=group)
    return dsq, idx, logP, status


def prob_sharded(ctx, O: torch.Tensor, logdet: torch.Tensor, patterns, precision="fx", group=None):
    """Exact log P of one batch evaluated by all ranks of a torch.distributed process group
    together (the strong-scaling split): rank k sweeps slice k of N of the batch's work
    units with ctx.prob_partial (equal unit counts, a large pattern cut by its subset
    prefix where the slices fall), one all_gather exchanges the slices' per-pattern
    partial sums (24 bytes and one flag per pattern and rank), and every rank combines
    them in rank order with ctx.prob_combine, so every rank holds the same result,
    bit for bit.  Without an initialised process group it is the one-rank case."""
    import torch.distributed as dist
    dist_on = dist.is_available() and dist.is_initialized()
    world = dist.get_world_size(group) if dist_on else 1
    rank = dist.get_rank(group) if dist_on else 0
    partial, pflag = ctx.prob_partial(O, patterns, rank, world, precision=precision)
    if world > 1:
        parts = [torch.empty_like(partial) for _ in range(world)]
        flags = [torch.empty_like(pflag) for _ in range(world)]
        dist.all_gather(parts, partial, group=group)
        dist.all_gather(flags, pflag, group=group)
        partials, pflags = torch.stack(parts), torch.stack(flags)
    else:
        partials, pflags = partial[None], pflag[None]
    return ctx.prob_combine(logdet, patterns, partials, pflags, precision=precision)


def patterns_numpy(t: torch.Tensor) -> np.ndarray:
    """(n, 2) uint64 numpy array from a device pattern tensor."""
    return t.detach().cpu().numpy().view(np.uint64)


def _clements_state(r, eta, theta, phi, gbs: "Context"):
    """Mesh unitary and state build on the device: (rd, Ud, state dict)."""
    M = r.shape[0]
    Ud = gbs.clements_unitary(theta, phi, M)
    rd = r.detach().to(device=gbs.device, dtype=torch.float64).contiguous()
    st = gbs.build_state(torch.view_as_complex(Ud.view(M, M, 2)), rd, float(eta), check=False)
    return rd, Ud, st


def _clements_chain(fctx, dsq):
    """(dr, deta, dtheta, dphi) from dL/dsigma_Q through the state build and the mesh."""
    rd, theta, phi, Ud, _, _ = fctx.saved_tensors
    gbs = fctx.gbs
    dU, dr, deta = gbs.grad_params(Ud, rd, fctx.eta, dsq)
    dth, dph = gbs.clements_grad(theta, phi, Ud, dU)
    return dr, deta[0], dth, dph


class LogProbClements(torch.autograd.Function):
    """log P of click patterns as a differentiable function of the squeezing r,
    the transmission eta and the mesh phases (theta, phi).  Forward: mesh
    unitary, state build and the exact sweep in libgbs (fixed point; double-double
    for patterns outside its range); backward: the double-double adjoint
    (gbs_grad), the state-build chain (gbs_grad_params) and the reverse pass
    through the mesh (gbs_clements_grad).

        logP = LogProbClements.apply(r, eta, theta, phi, patterns, ctx)
    """

    @staticmethod
    def forward(fctx, r, eta, theta, phi, patterns, gbs: Context):
        rd, Ud, st = _clements_state(r, eta, theta, phi, gbs)
        # fixed point, double-double for the patterns outside its range (in the library)
        out = gbs.prob(st["O"], st["logdet"], patterns, order=0, precision="auto")
        fctx.save_for_backward(rd, theta.detach(), phi.detach(), Ud, st["O"], st["logdet"])
        fctx.gbs, fctx.eta, fctx.patterns = gbs, float(eta), patterns
        return out["logP"]

    @staticmethod
    def backward(fctx, grad_logP):
        O, logdet = fctx.saved_tensors[4], fctx.saved_tensors[5]
        dsq, _, _ = fctx.gbs.grad(O, logdet, fctx.patterns, grad_logP.detach())
        return (*_clements_chain(fctx, dsq), None, None)


class LogProbClementsApprox(torch.autograd.Function):
    """As LogProbClements with the order-j moment approximation of log P (FP64
    minors) in the forward and its adjoint (gbs_grad_approx) in the backward: for
    patterns beyond the exact adjoint's 24 clicks.

        logP = LogProbClementsApprox.apply(r, eta, theta, phi, patterns, ctx, order)
    """

    @staticmethod
    def forward(fctx, r, eta, theta, phi, patterns, gbs: Context, order: int):
        rd, Ud, st = _clements_state(r, eta, theta, phi, gbs)
        out = gbs.prob(st["O"], st["logdet"], patterns, order=order, precision="fp64")
        fctx.save_for_backward(rd, theta.detach(), phi.detach(), Ud, st["O"], st["logdet"])
        fctx.gbs, fctx.eta, fctx.patterns, fctx.order = gbs, float(eta), patterns, int(order)
        return out["logP"]

    @staticmethod
    def backward(fctx, grad_logP):
        O, logdet = fctx.saved_tensors[4], fctx.saved_tensors[5]
        dsq, _, _ = fctx.gbs.grad_approx(O, logdet, fctx.patterns, grad_logP.detach(), fctx.order)
        return (*_clements_chain(fctx, dsq), None, None, None)
