"""Seeded synthetic inputs for Gaussian boson sampling workloads.

This module holds no part of the probability computation.  It only makes the
inputs that both the CUDA library and the FP64 oracle are run on:

* ``philox4x32_10``  -- the counter-based generator of Salmon, Moraes, Dror and
  Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11), written from its
  published definition.  The CUDA pattern generator implements the same
  function on the device; the two must agree bit for bit.
* ``haar_unitary``   -- Haar-random U by the QR method with phase fix
  (Mezzadri, "How to generate random matrices from the classical compact
  groups", 2007), normals by Box-Muller from Philox words.
* ``clements_unitary`` -- U from a rectangular mesh of M(M-1)/2 two-mode cells
  (Clements et al., Optica 3, 1460 (2016)), identity output phase screen.
* ``squeezing``      -- r_i ~ U[lo, hi] on the first K inputs, 0 elsewhere.
* ``gen_patterns``   -- click patterns: n ~ U{n_lo..n_hi}, then a uniform
  n-subset of the M detectors by a partial Fisher-Yates shuffle.

Conventions shared with the library: a_out = U a_in, so ``U[i, j]`` is the
amplitude from input j to output i; a click pattern is a pair of uint64 words
(bit i of word i // 64 set <=> detector i clicked), M <= 128.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "philox4x32_10", "philox_words", "uniform01", "normals", "haar_unitary",
    "clements_unitary", "clements_phases", "squeezing", "gen_patterns",
    "all_patterns", "pattern_modes", "modes_to_pattern", "Config", "CONFIGS", "accuracy_study",
    "STREAM_U", "STREAM_R", "STREAM_PATTERNS", "STREAM_ANCHORS",
]

# Stream ids (counter word 2) for the independent draws of one workload.
STREAM_U, STREAM_R, STREAM_PATTERNS, STREAM_ANCHORS = 0, 1, 2, 3

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr: np.ndarray, key) -> np.ndarray:
    """Philox4x32 with 10 rounds.

    ``ctr``: (..., 4) uint32 counters; ``key``: two uint32 words.  One round
    maps (c0, c1, c2, c3) to (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2),
    hi(M0*c0) ^ c3 ^ k1, lo(M0*c0)); the key is bumped by the Weyl constants
    between rounds.
    """
    c = np.asarray(ctr, dtype=np.uint64).copy()
    k0, k1 = int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF
    c0, c1, c2, c3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    for rnd in range(10):
        if rnd:
            k0 = (k0 + _W0) & 0xFFFFFFFF
            k1 = (k1 + _W1) & 0xFFFFFFFF
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1,
                          hi0 ^ c3 ^ np.uint64(k1), lo0)
    out = np.stack([c0, c1, c2, c3], axis=-1)
    return (out & _MASK32).astype(np.uint32)


def _key(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return (seed & 0xFFFFFFFF, seed >> 32)


def philox_words(seed: int, stream: int, index: np.ndarray, nwords: int) -> np.ndarray:
    """``nwords`` uint32 words for each item ``index`` of ``stream``.

    Item i draws its words from counters (i, block, stream, 0), block = 0, 1, ...
    (four words per block, in order).
    """
    index = np.asarray(index, dtype=np.uint64).reshape(-1)
    nblk = (nwords + 3) // 4
    ctr = np.zeros((index.size, nblk, 4), dtype=np.uint64)
    ctr[:, :, 0] = index[:, None]
    ctr[:, :, 1] = np.arange(nblk, dtype=np.uint64)[None, :]
    ctr[:, :, 2] = np.uint64(stream)
    w = philox4x32_10(ctr, _key(seed)).reshape(index.size, nblk * 4)
    return w[:, :nwords]


def uniform01(words: np.ndarray) -> np.ndarray:
    """Map uint32 words to doubles in (0, 1): (w + 0.5) / 2^32."""
    return (words.astype(np.float64) + 0.5) * (1.0 / 4294967296.0)


def normals(seed: int, stream: int, count: int) -> np.ndarray:
    """``count`` standard normals by Box-Muller on consecutive word pairs."""
    npairs = (count + 1) // 2
    w = philox_words(seed, stream, np.arange(npairs), 2)
    u1, u2 = uniform01(w[:, 0]), uniform01(w[:, 1])
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.stack([rad * np.cos(2.0 * np.pi * u2), rad * np.sin(2.0 * np.pi * u2)], axis=1)
    return z.reshape(-1)[:count]


def haar_unitary(M: int, seed: int, stream: int = STREAM_U) -> np.ndarray:
    """Haar-random M x M unitary (complex Gaussian QR with phase fix)."""
    g = normals(seed, stream, 2 * M * M).reshape(M, M, 2)
    z = (g[..., 0] + 1j * g[..., 1]) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))[None, :]


def clements_phases(M: int, seed: int, stream: int = STREAM_U):
    """theta, phi ~ U[0, 2 pi) for the M(M-1)/2 cells of the mesh."""
    ncell = M * (M - 1) // 2
    w = philox_words(seed, stream, np.arange(ncell), 2)
    return 2.0 * np.pi * uniform01(w[:, 0]), 2.0 * np.pi * uniform01(w[:, 1])


def clements_cells(M: int):
    """Mode pair (m, m+1) of every cell, in the order the cells act.

    Layer l = 0..M-1 holds the pairs whose first mode m has the parity of l.
    """
    cells = []
    for layer in range(M):
        for m in range(layer % 2, M - 1, 2):
            cells.append(m)
    assert len(cells) == M * (M - 1) // 2
    return cells


def clements_unitary(M: int, theta: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """U = T_last ... T_1 with T(theta, phi) on modes (m, m+1):
    [[e^{i phi} cos theta, -sin theta], [e^{i phi} sin theta, cos theta]]."""
    U = np.eye(M, dtype=np.complex128)
    for c, m in enumerate(clements_cells(M)):
        ct, st, e = math.cos(theta[c]), math.sin(theta[c]), complex(math.cos(phi[c]), math.sin(phi[c]))
        rows = U[[m, m + 1], :].copy()
        U[m, :] = e * ct * rows[0] - st * rows[1]
        U[m + 1, :] = e * st * rows[0] + ct * rows[1]
    return U


def squeezing(M: int, K: int, lo: float, hi: float, seed: int, stream: int = STREAM_R) -> np.ndarray:
    """r_i ~ U[lo, hi] for inputs i < K, r_i = 0 (vacuum) for i >= K."""
    r = np.zeros(M)
    if K:
        w = philox_words(seed, stream, np.arange(K), 1)[:, 0]
        r[:K] = lo + (hi - lo) * uniform01(w)
    return r


def _range32(word: np.ndarray, span) -> np.ndarray:
    """floor(word * span / 2^32): integer range reduction to [0, span)."""
    return ((word.astype(np.uint64) * np.asarray(span, dtype=np.uint64)) >> np.uint64(32)).astype(np.int64)


def gen_patterns(seed: int, M: int, n_lo: int, n_hi: int, n_pat: int,
                 stream: int = STREAM_PATTERNS) -> np.ndarray:
    """(n_pat, 2) uint64 click patterns.

    Pattern i uses words w_0, w_1, ... of item i: n = n_lo + range(w_0, n_hi-n_lo+1);
    then for k = 0..n-1: j = k + range(w_{k+1}, M-k), swap perm[k], perm[j];
    the clicked set is perm[0..n-1] (perm starts as the identity).
    """
    assert 1 <= M <= 128 and 0 <= n_lo <= n_hi <= M
    w = philox_words(seed, stream, np.arange(n_pat), n_hi + 1)
    out = np.zeros((n_pat, 2), dtype=np.uint64)
    for i in range(n_pat):
        n = n_lo + int(_range32(w[i, 0], n_hi - n_lo + 1))
        perm = list(range(M))
        for k in range(n):
            j = k + int(_range32(w[i, k + 1], M - k))
            perm[k], perm[j] = perm[j], perm[k]
        out[i] = modes_to_pattern(perm[:n])
    return out


def modes_to_pattern(modes) -> np.ndarray:
    lo = hi = 0
    for m in modes:
        m = int(m)
        if m < 64:
            lo |= 1 << m
        else:
            hi |= 1 << (m - 64)
    return np.array([lo, hi], dtype=np.uint64)


def pattern_modes(pat) -> list:
    """Ascending detector indices of a click pattern."""
    lo, hi = int(pat[0]), int(pat[1])
    return [i for i in range(64) if lo >> i & 1] + [64 + i for i in range(64) if hi >> i & 1]


def all_patterns(M: int) -> np.ndarray:
    """All 2^M patterns, pattern index = bitmask (M <= 24)."""
    assert M <= 24
    idx = np.arange(1 << M, dtype=np.uint64)
    return np.stack([idx, np.zeros_like(idx)], axis=1)


@dataclass
class Config:
    """One synthetic workload: device, state and patterns."""
    name: str
    M: int
    K: int
    r_lo: float
    r_hi: float
    eta: float
    interferometer: str          # "haar" or "clements"
    seed: int
    n_lo: int = 0
    n_hi: int = 0
    n_pat: int = 0
    orders: tuple = (0,)
    exact_n_max: int = 64
    anchors: int = 0
    anchor_n: int = 0
    note: str = ""

    def unitary(self) -> np.ndarray:
        if self.interferometer == "haar":
            return haar_unitary(self.M, self.seed)
        th, ph = clements_phases(self.M, self.seed)
        return clements_unitary(self.M, th, ph)

    def squeezing(self) -> np.ndarray:
        return squeezing(self.M, self.K, self.r_lo, self.r_hi, self.seed)

    def patterns(self) -> np.ndarray:
        if self.n_pat == 0:
            return all_patterns(self.M)
        return gen_patterns(self.seed, self.M, self.n_lo, self.n_hi, self.n_pat)

    def anchor_patterns(self) -> np.ndarray:
        return gen_patterns(self.seed, self.M, self.anchor_n, self.anchor_n, self.anchors,
                            stream=STREAM_ANCHORS)


# The five benchmark workloads, and the 30-mode device shape of the paper's click-number
# figures (15 inputs squeezed r = 1.4, lossless).  Seeds: workload c uses seed c (the
# 8-mode one uses 0).
CONFIGS = {
    "m8_all": Config("m8_all", M=8, K=8, r_lo=0.8, r_hi=0.8, eta=1.0, interferometer="haar",
                     seed=0, note="all 256 patterns, sum must be 1"),
    "m24_exact": Config("m24_exact", M=24, K=12, r_lo=0.6, r_hi=1.2, eta=0.5,
                        interferometer="haar", seed=2, n_lo=12, n_hi=20, n_pat=1024),
    "m50_approx": Config("m50_approx", M=50, K=25, r_lo=0.8, r_hi=1.4, eta=0.4,
                         interferometer="haar", seed=3, n_lo=10, n_hi=40, n_pat=4096,
                         orders=(2, 3, 4), exact_n_max=22),
    "m32_grad": Config("m32_grad", M=32, K=16, r_lo=0.6, r_hi=1.2, eta=0.6,
                       interferometer="clements", seed=4, n_lo=8, n_hi=16, n_pat=512),
    "m100_approx": Config("m100_approx", M=100, K=50, r_lo=1.1, r_hi=1.6, eta=0.3,
                          interferometer="haar", seed=5, n_lo=40, n_hi=90, n_pat=16384,
                          orders=(2, 3, 4), exact_n_max=0, anchors=64, anchor_n=30),
    "m30_device": Config("m30_device", M=30, K=15, r_lo=1.4, r_hi=1.4, eta=1.0, interferometer="haar",
                         seed=6, note="whole-device p(n); the all-click point by orders 2-4"),
}


def accuracy_study():
    """The grid of the fourth-order accuracy study (the paper's Fig. 4): lossless devices with
    half of the inputs squeezed, Haar U, 100 uniformly random n-click outcomes per point.

    * ``vs_m``: r = 1.6, n in {6, 10, 14, 18, 22} clicks on M = round(n / f) modes for the
      clicked fractions f = 1/3, 1/2, 0.7 (n = 18 gives the paper's 54, 36 and 26 modes);
    * ``vs_r``: 20 clicks on 30 modes (15 inputs squeezed), r = 0.4 .. 2.0.

    Returns ``{"vs_m": [Config, ...], "vs_r": [Config, ...]}``; seeds 100 + point index.
    """
    vs_m, vs_r = [], []
    k = 0
    for frac, tag in ((1.0 / 3.0, "f33"), (0.5, "f50"), (0.7, "f70")):
        for n in (6, 10, 14, 18, 22):
            M = int(round(n / frac))
            vs_m.append(Config("acc_%s_n%d" % (tag, n), M=M, K=M // 2, r_lo=1.6, r_hi=1.6, eta=1.0,
                               interferometer="haar", seed=100 + k, n_lo=n, n_hi=n, n_pat=100,
                               orders=(4,), note="clicked fraction %.2f" % frac))
            k += 1
    for i in range(9):
        rr = round(0.4 + 0.2 * i, 1)
        vs_r.append(Config("acc_r%.1f" % rr, M=30, K=15, r_lo=rr, r_hi=rr, eta=1.0, interferometer="haar",
                           seed=100 + k, n_lo=20, n_hi=20, n_pat=100, orders=(4,)))
        k += 1
    return {"vs_m": vs_m, "vs_r": vs_r}
