"""FP64 oracle for the paper's moment approximation (test infrastructure only).

The steps follow Methods ("Partition function", "Probability of any sample",
"Moments calculation", "Approximation method"), extended to uniform loss by
the covariance form.  For a click pattern S with n modes:

1. Sectors (Methods, "Partition function"): for every sub-ensemble Z of S the
   generating function  Z_Z(t) = det(I - t O_Z)^{-1/2} = sum_k c_k[Z] t^k  has
   c_k[Z] det(sigma_Q)^{-1/2} = P(k photons in Z, vacuum on every other
   detector).  The paper's Fourier sum over nu is the coefficient extraction
   of this series; here the coefficients are computed exactly from the
   eigenvalues lambda of O_Z:  log Z_Z(t) = 1/2 sum_p (sum_i lambda_i^p) t^p / p,
   then the series exponential.
2. Moments (Methods, "Moments calculation"): in the sub-ensemble of S, let v
   be the number of detectors of S left in vacuum.  The minors with w
   detectors removed give the factorial moments of v in every sector,
        D_w^(k) = sum_{W subset S, |W| = w} c_k[S \\ W] = sum_v C(v, w) q_k(v),
   for w = 0..j; raw moments follow with Stirling numbers of the second kind.
3. Inverse moment problem (Methods, "Approximation method"): in each sector
   q_k(v) ~ exp(-f(v)) with f a polynomial of degree j whose moments 0..j
   match; solved as the convex maximum-entropy dual by damped Newton.
4. The all-clicked point v = 0 of every sector is summed:
        P(S) ~ det(sigma_Q)^{-1/2} sum_k exp(-f_k(0)).

Readings where the paper is silent:
* the fit variable is v = n - c (same polynomial family as the click count c);
* sector k >= 1 lives on v in [max(0, n-k), n-1]; sectors k < n add nothing;
* the polynomial degree is min(j, |support| - 1), so the fit is exact when
  the support has at most j + 1 points;
* "iteratively find parameters" is iterated to convergence of the parameters:
  after the moment residual reaches 1e-13 one more full Newton step is taken
  (the extrapolation to v = 0 is ill-conditioned, a residual alone leaves the
  last point uncertain); a fallback to a lower order is reported only when the
  sectors that fell back carry >= 1e-4 of the summed last points;
* x = v / n is the variable inside the Newton solve (conditioning only);
* the paper's discrete set of nu is a circle |t| = rho: rho is the Chernoff
  saddle for sector n, rho = argmin over the radii RHOS at which I -+ rho O_S
  stay positive definite (the largest excluded) of log Z_S(rho) - n log rho,
  so that the sectors carrying the all-clicked point sit near the peak of
  c_k rho^k (for improbable patterns they lie far in the upper tail);
* the sector sum stops at K_max, the first K whose tail sum_{k>K} c_k rho^k is
  below 1e-14 Z_S(rho);
* a sector whose tilted mass D_0^(k) rho^k is below eps_sector = 1e-12 of the
  largest contributes nothing: such sectors are rounding noise (e.g. the odd
  sectors of a lossless state, exactly zero).
"""
from __future__ import annotations

import math
from itertools import combinations

import numpy as np

TAIL_EPS = 1e-14
EPS_SECTOR = 1e-12
FLAG_SHARE = 1e-4
RHOS = (1.0, 1.02, 1.05, 1.1, 1.15, 1.2, 1.25, 1.3, 1.4, 1.5, 1.7, 2.0, 2.5, 3.0, 4.0)


def sub_rows(modes, M):
    """Row indices (x of each mode, then p of each mode) of a mode set in xp order."""
    modes = list(modes)
    return modes + [m + M for m in modes]


def series_coeffs(Osub: np.ndarray, K: int) -> np.ndarray:
    """c_0..c_K of det(I - t Osub)^{-1/2} (Osub real symmetric)."""
    c = np.zeros(K + 1)
    c[0] = 1.0
    if Osub.size == 0:
        return c
    lam = np.linalg.eigvalsh(Osub)
    a = np.zeros(K + 1)
    pw = np.ones_like(lam)
    for p in range(1, K + 1):
        pw = pw * lam
        a[p] = 0.5 * pw.sum() / p
    for k in range(1, K + 1):
        p = np.arange(1, k + 1)
        c[k] = np.dot(p * a[1:k + 1], c[k - p]) / k
    return c


def _pd_logdet(X: np.ndarray):
    """log det X if X is positive definite, else None."""
    try:
        L = np.linalg.cholesky(X)
    except np.linalg.LinAlgError:
        return None
    return 2.0 * np.log(np.diag(L)).sum()


def choose_tilt(O: np.ndarray, M: int, modes, rhos=RHOS) -> float:
    """rho = argmin_{rho in rhos, valid, not the largest valid} log Z_S(rho) - n log rho."""
    rows = sub_rows(modes, M)
    Os = O[np.ix_(rows, rows)]
    n = len(modes)
    if n == 0:
        return 1.0
    I = np.eye(len(rows))
    valid = []
    for rho in rhos:
        l_minus = _pd_logdet(I - rho * Os)
        if l_minus is None or (rho > 1.0 and _pd_logdet(I + rho * Os) is None):
            break
        valid.append((rho, -0.5 * l_minus))          # (rho, log Z_S(rho))
    cands = valid[:-1] if len(valid) > 1 else valid
    best = min(cands, key=lambda v: (v[1] - n * math.log(v[0]), v[0]))
    return best[0]


def choose_kmax(O: np.ndarray, M: int, modes, rho: float = 1.0) -> int:
    """Smallest K whose tail sum_{k>K} c_k rho^k is below TAIL_EPS Z_S(rho).

    The tail is summed from the series itself (every c_k rho^k is positive), far
    enough out that the terms left are below 1e-30 of Z_S(rho); Z_S(rho) minus a
    partial sum would cancel to the rounding of Z_S(rho), ~1e-16 relative, which is
    too close to TAIL_EPS to decide K reliably."""
    rows = sub_rows(modes, M)
    Os = O[np.ix_(rows, rows)] * rho
    if Os.size == 0:
        return 0
    total = np.linalg.det(np.eye(len(rows)) - Os) ** -0.5
    K = 64
    while True:
        c = series_coeffs(Os, K)
        if c[-1] < 1e-30 * total and c[-1] <= c[-2]:
            tail = np.cumsum(c[::-1])[::-1]            # tail[k] = sum_{k' >= k} c_k'
            return int(np.nonzero(tail[1:] < TAIL_EPS * total)[0][0])
        if K > 1 << 16:
            raise RuntimeError("sector series does not converge")
        K *= 2


def factorial_moment_tables(O: np.ndarray, M: int, modes, j: int, K: int,
                            rho: float = 1.0) -> np.ndarray:
    """D[w, k] rho^k with D[w, k] = sum over groups W of S with |W| = w of c_k[S \\ W], w = 0..j."""
    modes = list(modes)
    n = len(modes)
    D = np.zeros((j + 1, K + 1))
    for w in range(min(j, n) + 1):
        for W in combinations(range(n), w):
            keep = [modes[a] for a in range(n) if a not in W]
            rows = sub_rows(keep, M)
            D[w] += series_coeffs(rho * O[np.ix_(rows, rows)], K)
    return D


def stirling2(i: int, w: int) -> int:
    if i == w:
        return 1
    if w == 0 or w > i:
        return 0
    return w * stirling2(i - 1, w) + stirling2(i - 1, w - 1)


def raw_moments(Dk: np.ndarray, j: int) -> np.ndarray:
    """mu_i = sum_v v^i q(v) = sum_w S(i, w) w! D_w, i = 0..j."""
    return np.array([sum(stirling2(i, w) * math.factorial(w) * Dk[w] for w in range(i + 1))
                     for i in range(j + 1)])


def maxent_fit(support: np.ndarray, m: np.ndarray, tol: float = 1e-13, max_iter: int = 200,
               stall_accept: float = 1e3):
    """Coefficients a of q(x) = exp(-sum_i a_i x^i) on the support points x with
    sum_x x^i q(x) = m_i (i = 0..J, m_0 = 1).  Returns (a, converged).  A fit whose line
    search stalls stands if its residual is within stall_accept * tol."""
    J = m.size - 1
    X = np.vander(support, J + 1, increasing=True)            # X[s, i] = x_s^i
    a = np.zeros(J + 1)
    a[0] = math.log(support.size)

    def phi(a):
        return np.exp(-X @ a).sum() + a @ m

    f = phi(a)
    for it in range(max_iter):
        q = np.exp(-X @ a)
        g = m - X.T @ q
        H = (X * q[:, None]).T @ X
        try:
            step = np.linalg.solve(H, g)
        except np.linalg.LinAlgError:
            return a, bool(np.max(np.abs(g)) <= tol)
        if np.max(np.abs(g)) <= tol:
            # one last full Newton step: near the optimum it squares the error, so
            # the parameters (and the extrapolated q(0)) converge, not only the moments
            return a - step, True
        # gradient of phi is g; Newton direction -step; Armijo backtracking.
        # Near the optimum the decrease of phi is below its rounding, so a step
        # that halves the gradient is accepted as well.
        t = 1.0
        gmax = np.max(np.abs(g))
        while True:
            an = a - t * step
            fn = phi(an)
            if np.isfinite(fn) and fn <= f - 1e-4 * t * (g @ step):
                break
            if np.isfinite(fn) and fn <= f + 1e-14 * abs(f) and \
                    np.max(np.abs(m - X.T @ np.exp(-X @ an))) <= 0.5 * gmax:
                break
            t *= 0.5
            if t < 1e-12:
                # no further decrease: the moments sit on the boundary of the moment
                # cone (a support point of vanishing weight) up to their rounding;
                # the fit stands if the residual is at that level
                return a, bool(gmax <= stall_accept * tol)
        a, f = an, fn
    q = np.exp(-X @ a)
    return a, bool(np.max(np.abs(m - X.T @ q)) <= stall_accept * tol)


def sector_fit(Dk: np.ndarray, n: int, k: int, j: int, stall_accept: float = 1e3):
    """The fit behind sector_last_point: (value, flag, a, J) with a the coefficients of
    the normalised fit exp(-sum_i a_i x^i), x = v / n, of degree J (None when no fit)."""
    if k < n or Dk[0] <= 0.0:
        return 0.0, 0, None, -1
    if n == 0:
        return Dk[0], 0, None, -1
    v = np.arange(max(0, n - k), n, dtype=np.float64)          # v = n is empty for k >= 1
    Jmax = min(j, v.size - 1)
    mu = raw_moments(Dk, Jmax)
    x = v / n
    for J in range(Jmax, -1, -1):
        mnorm = np.array([mu[i] / n ** i for i in range(J + 1)]) / mu[0]
        a, ok = maxent_fit(x, mnorm, stall_accept=stall_accept)
        if ok:
            return mu[0] * math.exp(-a[0]), 0 if J == Jmax else 1, a, J
    return 0.0, 2, None, -1


def sector_last_point(Dk: np.ndarray, n: int, k: int, j: int, stall_accept: float = 1e3):
    """Estimate of q_k(v = 0) from the factorial moments D_0..D_j of sector k.

    Returns (value, flag) with flag 0 = fitted at order j' = min(j, |V|-1),
    1 = fell back to a lower order, 2 = no fit possible (value 0)."""
    val, flag, _, _ = sector_fit(Dk, n, k, j, stall_accept)
    return val, flag


def logprob_from_tables(D: np.ndarray, n: int, j: int, rho: float, logdet_sigmaQ: float,
                        eps_sector: float = EPS_SECTOR, flag_share: float = FLAG_SHARE,
                        stall_accept: float = 1e3):
    """Steps 3 and 4 from the tilted moment tables D[w, k] = D_w^(k) rho^k: each sector's
    fit, its all-clicked point, and their sum.  Returns (logP, parts, flag)."""
    K = D.shape[1] - 1
    parts = np.zeros(K + 1)                                  # tilted last points
    fell = np.zeros(K + 1, dtype=bool)
    floor = eps_sector * D[0].max()
    for k in range(K + 1):
        if D[0, k] < floor:
            continue
        val, fl = sector_last_point(D[:, k], n, k, j, stall_accept)
        parts[k] = val
        fell[k] = fl > 0
    # sum_k parts[k] rho^{-k}, in logs (rho^{-k} can leave the double range)
    nz = np.nonzero(parts > 0)[0]
    flags = 0
    if nz.size:
        lg = np.log(parts[nz]) - nz * math.log(rho)
        top = lg.max()
        w = np.exp(lg - top)
        logsum = top + math.log(w.sum())
        # a fallback is reported when the sectors that fell back carry >= FLAG_SHARE of the sum
        if w[fell[nz]].sum() >= flag_share * w.sum():
            flags = 1
    else:
        logsum = -math.inf
    return -0.5 * logdet_sigmaQ + logsum, parts, flags


def approx_logprob(O: np.ndarray, logdet_sigmaQ: float, M: int, modes, j: int,
                   K: int | None = None, eps_sector: float = EPS_SECTOR, rho: float | None = None,
                   rhos=RHOS, flag_share: float = FLAG_SHARE, stall_accept: float = 1e3):
    """log P(S) by the order-j approximation.  Returns (logP, info dict).  K and rho
    default to choose_kmax and choose_tilt (over the radii rhos); fixing them makes log P
    a smooth function of O (for derivatives by differences).  eps_sector, flag_share and
    stall_accept are the readings' constants (the tests vary them to show log P does not
    depend on them)."""
    modes = list(modes)
    n = len(modes)
    if rho is None:
        rho = choose_tilt(O, M, modes, rhos)
    if K is None:
        K = choose_kmax(O, M, modes, rho)
    D = factorial_moment_tables(O, M, modes, j, K, rho)     # tilted: D_w^(k) rho^k
    logP, parts, flags = logprob_from_tables(D, n, j, rho, logdet_sigmaQ, eps_sector, flag_share, stall_accept)
    return logP, dict(K=K, D=D, parts=parts, flag=flags, rho=rho)


def exact_sector_last_points(O: np.ndarray, M: int, modes, K: int) -> np.ndarray:
    """Exact q_k(v = 0) = sum_{Z subset S} (-1)^{n-|Z|} c_k[Z], by inclusion-exclusion
    inside each sector (small n only)."""
    modes = list(modes)
    n = len(modes)
    out = np.zeros(K + 1)
    for z in range(1 << n):
        Z = [modes[a] for a in range(n) if z >> a & 1]
        rows = sub_rows(Z, M)
        sgn = -1.0 if (n - len(Z)) & 1 else 1.0
        out += sgn * series_coeffs(O[np.ix_(rows, rows)], K)
    return out


def sector_distribution(O: np.ndarray, logdet_sigmaQ: float, M: int, K: int) -> np.ndarray:
    """Whole-device sectors p_k(n), k = 0..K, n = 0..M (Results, "Calculation of sectors"):
    the probability of n clicks with k photons, summed over every pattern S with n clicks
    of P(S, k) = det(sigma_Q)^{-1/2} q_k(S), q_k(S) the inclusion-exclusion of the sector
    coefficients over the subsets of S (exact_sector_last_points).  All 2^M patterns:
    small M only."""
    out = np.zeros((K + 1, M + 1))
    for mask in range(1 << M):
        modes = [i for i in range(M) if mask >> i & 1]
        out[:, len(modes)] += exact_sector_last_points(O, M, modes, K)
    return out * math.exp(-0.5 * logdet_sigmaQ)


def sector_curve(Dk: np.ndarray, n: int, k: int, j: int):
    """The order-j estimate of sector k's whole distribution q_k(v), v = 0..n, from its
    factorial moments D_0..D_j (Results, "Approximation scheme": exp(-f_j) fitted to the
    moments on the sector's support v in [max(0, n-k), n-1]; k = 0 is v = n alone).
    Returns (q, flag) with the flags of sector_last_point."""
    q = np.zeros(n + 1)
    if Dk[0] <= 0.0:
        return q, 0
    if k == 0 or n == 0:
        q[n] = Dk[0] if k == 0 else 0.0
        return q, 0
    v = np.arange(max(0, n - k), n, dtype=np.float64)
    Jmax = min(j, v.size - 1)
    mu = raw_moments(Dk, Jmax)
    x = v / n
    for J in range(Jmax, -1, -1):
        mnorm = np.array([mu[i] / n ** i for i in range(J + 1)]) / mu[0]
        a, ok = maxent_fit(x, mnorm)
        if ok:
            q[v.astype(int)] = mu[0] * np.exp(-np.vander(x, J + 1, increasing=True) @ a)
            return q, 0 if J == Jmax else 1
    return q, 2


def approx_sector_curves(O: np.ndarray, logdet_sigmaQ: float, M: int, modes, j: int, K: int):
    """Every sector's fitted distribution for the pattern S (the tilt and sector range of
    approx_logprob): out[k, c] = det(sigma_Q)^{-1/2} rho^-k q_k(v = n - c), k = 0..K."""
    modes = list(modes)
    n = len(modes)
    rho = choose_tilt(O, M, modes)
    Kmax = choose_kmax(O, M, modes, rho)
    D = factorial_moment_tables(O, M, modes, j, Kmax, rho)
    floor = EPS_SECTOR * D[0].max()
    out = np.zeros((K + 1, n + 1))
    for k in range(min(K, Kmax) + 1):
        if D[0, k] < floor:
            continue
        q, _ = sector_curve(D[:, k], n, k, j)
        out[k] = q[::-1] * math.exp(-0.5 * logdet_sigmaQ - k * math.log(rho))
    return out


# ---- gradient of the approximation (not in the paper) -----------------------------
# log P = -1/2 log det sigma_Q + log sum_k part_k rho^-k, part_k the fitted last point of
# sector k.  Reverse mode, step by step:
#  * the sum:   d/d part_k = rho^-k / sum_k' part_k' rho^-k';
#  * the fit:   the unnormalised fit F(x) = exp(-sum_i b_i x^i) matches the moments
#               mu'_i = mu_i / n^i on its support, so by implicit differentiation of
#               sum_s x_s^i F(x_s) = mu'_i,  d F(0) = F(0) (H^-1 d mu')_0 with
#               H_il = sum_s x_s^(i+l) F(x_s); with the normalised fit of coefficients a
#               (F = mu_0 exp(-sum a_i x^i)) that is  d part / d mu'_i = e^-a_0 (Hn^-1)_0i;
#  * moments:   mu'_i = sum_{w <= i} S(i, w) w! D_w / n^i;
#  * sectors:   D_w^(k) = sum_{|W| = w} c_k[rho O_{S \ W}], and for a real symmetric X
#               d c_k[X] / dX = 1/2 sum_{m < k} c_{k-1-m} X^m  (the t^k coefficient of
#               d det(I - t X)^-1/2 / dX = 1/2 t Z(t) (I - t X)^-1), evaluated on the
#               eigenvectors of X;
#  * O = I - A:  d / dA_S = -d / dO_S.

def fit_last_point_adjoint(n: int, a: np.ndarray, J: int, jmax: int) -> np.ndarray:
    """d part / d D_w, w = 0..jmax, of a sector fitted on v = 0..n-1 at degree J."""
    x = np.arange(n, dtype=np.float64) / n
    X = np.vander(x, J + 1, increasing=True)
    q = np.exp(-X @ a)
    Hn = (X * q[:, None]).T @ X
    e0 = np.zeros(J + 1)
    e0[0] = 1.0
    y = np.linalg.solve(Hn, e0)                    # row 0 of Hn^-1 (Hn symmetric)
    beta = np.zeros(jmax + 1)
    for w in range(J + 1):
        beta[w] = math.exp(-a[0]) * sum(y[i] * stirling2(i, w) * math.factorial(w) / n ** i
                                        for i in range(w, J + 1))
    return beta


def series_coeffs_adjoint(X: np.ndarray, gam: np.ndarray) -> np.ndarray:
    """sum_k gam_k d c_k[X] / dX for X real symmetric, k = 0..len(gam)-1."""
    K = gam.size - 1
    lam, Q = np.linalg.eigh(X)
    c = series_coeffs(X, K)
    # r_m = sum_{k > m} gam_k c_{k-1-m};  h(lambda) = 1/2 sum_m r_m lambda^m
    r = np.array([np.dot(gam[m + 1:], c[:K - m]) for m in range(K)])
    h = np.zeros_like(lam)
    for m in range(K - 1, -1, -1):
        h = h * lam + r[m]
    return 0.5 * (Q * h[None, :]) @ Q.T


def approx_logprob_grad(O: np.ndarray, logdet_sigmaQ: float, M: int, modes, j: int,
                        K: int | None = None, rho: float | None = None):
    """(log P, dlog P / dA_S) of the order-j approximation, A = I - O; the second is
    2n x 2n in the row order of sub_rows(modes) and excludes the -1/2 log det sigma_Q
    term (which depends on sigma_Q, not on A_S)."""
    modes = list(modes)
    n = len(modes)
    logP, info = approx_logprob(O, logdet_sigmaQ, M, modes, j, K=K, rho=rho)
    grad = np.zeros((2 * n, 2 * n))
    if n == 0 or not np.isfinite(logP):
        return logP, grad
    rho, K, D = info["rho"], info["K"], info["D"]
    logsum = logP + 0.5 * logdet_sigmaQ
    floor = EPS_SECTOR * D[0].max()
    gam = np.zeros((j + 1, K + 1))                 # d log sum / d D[w, k] (tilted tables)
    for k in range(K + 1):
        if D[0, k] < floor:
            continue
        val, _, a, J = sector_fit(D[:, k], n, k, j)
        if val <= 0.0 or a is None:
            continue
        g = math.exp(-k * math.log(rho) - logsum)
        gam[:, k] = g * fit_last_point_adjoint(n, a, J, j)
    for w in range(min(j, n) + 1):
        if not gam[w].any():
            continue
        for W in combinations(range(n), w):
            keep = [a for a in range(n) if a not in W]
            loc = keep + [a + n for a in keep]      # local rows of S \\ W (x block, p block)
            rows = sub_rows([modes[a] for a in keep], M)
            dX = series_coeffs_adjoint(rho * O[np.ix_(rows, rows)], gam[w])
            grad[np.ix_(loc, loc)] -= rho * dX
    return logP, grad
