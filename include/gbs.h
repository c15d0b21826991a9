/*
 * gbs.h -- C ABI of libgbs: click-pattern probabilities of a Gaussian boson
 * sampler with threshold detectors, on one NVIDIA GB300 (sm_103a).
 *
 * Method: Popova & Rubtsov, "Cracking the Quantum Advantage threshold for
 * Gaussian Boson Sampling" (arXiv 2106.01445).  Section names below refer to
 * that paper.
 *
 * Conventions shared by every entry point
 *  - M modes, 1 <= M <= 128.  a_out = U a_in: U[i*M + j] is the amplitude from
 *    input j to output (detector) i.  Complex arrays are interleaved (re, im).
 *  - Quadratures in xp order (x_1..x_M, p_1..p_M), hbar = 1, vacuum sigma = I/2.
 *    Every 2M x 2M matrix is row-major FP64.
 *  - A click pattern is two uint64 words: bit i of word i/64 set <=> detector i
 *    clicked.
 *  - Pointers are DEVICE pointers unless the name ends in _host.  The caller
 *    owns every buffer passed in; the context owns its workspace.
 *  - Calls are asynchronous on the context's stream unless stated otherwise.
 *    They return a gbs_status; a non-zero code leaves outputs undefined and
 *    gbs_last_error() describes it.  Per-pattern problems are reported in the
 *    per-pattern status array and never fail the batch.
 *  - No entry point aborts, traps or waits without a bound.
 */
#ifndef GBS_H
#define GBS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gbs_ctx gbs_ctx;

typedef enum {
    GBS_OK = 0,
    GBS_E_INVALID = 1,     /* bad argument (size, range, pointer, non-unitary U) */
    GBS_E_CUDA = 2,        /* a CUDA runtime call failed */
    GBS_E_NOMEM = 3,       /* workspace too small (reserve more) or allocation failed */
    GBS_E_NONPOSITIVE = 4, /* signed sum T <= its error bound: log P undefined */
    GBS_E_NOT_SPD = 5,     /* a pivot of an SPD factorisation was not positive */
    GBS_E_TIMEOUT = 6,     /* reserved: no entry point of this version returns it.  Every device
                              loop here is bounded by its own work count (persistent loops end
                              when their ticket passes the unit count; Newton fits stop after a
                              fixed number of steps and report GBS_E_FIT), and no kernel waits
                              on another */
    GBS_E_FIT = 7,         /* approximation: a sector fit fell back to a lower order */
    GBS_E_RANGE = 8,       /* GBS_FX: a pivot determinant below 2^-8 or an entry of O beyond
                              4 left the fixed-point range (evaluate in GBS_DD instead) */
    GBS_E_FLOOR = 9        /* approximation with FP32 minors: sectors below the FP32 noise floor
                              (1e-6 of the largest tilted sector) could carry 1e-4 or more of the
                              estimate, which FP32 moments cannot resolve; logP is returned but
                              unreliable: evaluate with GBS_FF or GBS_FP64 instead */
} gbs_status;

typedef enum {
    GBS_FP64 = 0,        /* every factorisation and sum in FP64 */
    GBS_FP32_SPLIT = 1,  /* subset factorisations in FP32; signed sum compensated, FP64 result */
    GBS_DD = 2,          /* double-double (~106-bit) factorisations and sum, on the FP64 pipes:
                            for patterns whose signed sum cancels beyond FP64 (kappa u64 >~ 1e-10) */
    GBS_FX = 3,          /* exact sum only: 128-bit fixed-point (Q16.112) factorisations on the
                            integer pipes, double-double prefactors and sum; accuracy as GBS_DD
                            (~2^-100 per term) at a fraction of its cost.  Needs every pivot
                            determinant of the Schur recursion >= 2^-8 (true when the largest
                            eigenvalue of sigma_Q is below 16); else GBS_E_RANGE */
    GBS_FF = 4,          /* approximation only: float-float (~48-bit) complex minors on the FP32
                            pipes; FP64-class moments at a fraction of FP64's cost (n <= 79) */
    GBS_AUTO = 5,        /* exact sum: GBS_FX, then GBS_DD for the patterns it reports GBS_E_RANGE,
                            then GBS_FX192 for the valid results whose err_bound exceeds 1e-10 (on
                            the device, no host synchronisation; gbs_reserve covers it; a batch
                            that needs neither rerun costs two sweeps over no units);
                            approximation: GBS_FF */
    GBS_FX192 = 6        /* exact sum only: 192-bit fixed point (Q16.176), prefactors and sums as
                            192-bit mantissas with exponents, unit sums added exactly per pattern:
                            per-term error ~2^-164 for signed sums that cancel beyond what
                            GBS_FX and GBS_DD resolve (kappa ~1e20 and more; err_bound says when
                            they do not suffice).  Same range condition as GBS_FX (GBS_E_RANGE).
                            Not taken by gbs_prob_noalloc or gbs_prob_partial */
} gbs_precision;

/* ---- context ------------------------------------------------------------ */

/* Create a context on CUDA device `device` issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  Errors: GBS_E_INVALID,
 * GBS_E_CUDA. */
int gbs_create(gbs_ctx **ctx, int device, void *cuda_stream);
int gbs_destroy(gbs_ctx *ctx);
int gbs_set_stream(gbs_ctx *ctx, void *cuda_stream);
/* Last error message of this context (static storage owned by the context). */
const char *gbs_last_error(const gbs_ctx *ctx);
/* Library version as major*10000 + minor*100 + patch. */
int gbs_version(void);

/* Pre-size the workspace for up to n_pat patterns of up to n_max clicks so
 * that later gbs_prob calls within those limits allocate nothing and never
 * synchronise (needed for CUDA-graph capture).  Synchronous.  The reservation
 * covers the exact sum (order 0).  The approximation, the whole-device
 * distributions and the gradients may grow the context's buffers, which frees
 * the ones a graph captured earlier refers to: capture after such calls, or make
 * them on a second context. */
int gbs_reserve(gbs_ctx *ctx, int n_pat, int n_max);

/* Autotuner (not in the paper): runs the exact sweep of these patterns with every
 * split s = 0..3 of a work unit (the prefix modes a CTA loops over inside one unit:
 * 2^(s + 9 or 10) subsets per unit) and keeps the fastest for this precision in the
 * context; later gbs_prob, gbs_reserve and gbs_prob_noalloc calls use it.  Choose
 * it before gbs_reserve (a reservation sized for one split may not hold a finer
 * one: such splits are skipped).  Allocates scratch for its outputs and
 * synchronises: not for use under stream capture.  best_split / best_ms (mean ms of
 * one sweep) may be NULL.  Errors: GBS_E_INVALID, GBS_E_CUDA, GBS_E_NOMEM. */
int gbs_autotune(gbs_ctx *ctx, int M, const double *O, const double *logdet_sigmaQ,
                 const uint64_t *patterns, int n_pat, int precision, int *best_split, double *best_ms);

/* ---- state build (Methods, "Model" and "Partition function") ------------
 * From U (M x M complex, unitary), squeezing r (M, r_j = 0 for vacuum
 * inputs) and uniform transmission eta in (0, 1]:
 *   sigma   = eta R sigma_in R^T + (1 - eta) I/2,  R = [[Re U, -Im U], [Im U, Re U]],
 *   sigma_in = diag(e^{-2r}/2 (x), e^{2r}/2 (p)),
 *   sigma_Q = sigma + I/2,  O = I - sigma_Q^{-1},  logdet = log det sigma_Q.
 * sigma may be NULL.  logdet_sigmaQ points to one double on the device.
 * status_dev: optional device int32 receiving GBS_OK or GBS_E_INVALID (U not
 * unitary to 1e-10, r < 0 or not finite); if NULL the call synchronises and
 * returns that status itself. */
int gbs_build_state(gbs_ctx *ctx, int M, const double *U, const double *r, double eta,
                    double *sigma, double *O, double *logdet_sigmaQ, int32_t *status_dev);

/* ---- click-pattern probabilities ---------------------------------------
 * Methods, "Probability of any sample" and Eq. (p(n)):
 *   P(S) = det(sigma_Q)^{-1/2} sum_{Z subset S} (-1)^{|S|-|Z|} det(I - O_Z)^{-1/2},
 * O_Z = rows/columns x and p of the modes in Z.
 * order 0: the exact sum over all 2^n subsets (n <= 40).
 * order j = 1..4 (the paper uses 2..4): the moment approximation (Methods,
 *   "Partition function", "Moments calculation", "Approximation method"):
 *   sector tables of the minors removing <= j detectors at t = e^{i nu} (nu on
 *   L points, L - 1 a bound on the sector index with tail < 1e-14), inverse
 *   DFT, per-sector maximum-entropy fit of moments 0..j, sum of the all-clicked
 *   points.  Order 0 takes GBS_FP64, GBS_FP32_SPLIT, GBS_DD, GBS_FX and GBS_AUTO (GBS_FX,
 *   then GBS_DD for its out-of-range patterns); order > 0 takes GBS_FF (float-float complex
 *   minors, n <= 79; also GBS_AUTO), GBS_FP64 (n <= 79) or GBS_FP32_SPLIT (FP32 complex
 *   minors, FP64 sums and fits; n <= 112).  For order > 0, kappa returns the
 *   sector bound K, err_bound is NaN, and status GBS_E_FIT marks a pattern where
 *   some sector fit fell back to a lower order (logP is still returned).
 * Inputs: O (2M x 2M), logdet_sigmaQ (device, one double), patterns (n_pat x 2
 * uint64).  Outputs per pattern (each may be NULL except logP):
 *   logP      natural log of P(S)
 *   kappa     condition number sum_Z |term| / |T| of the signed sum (order 0)
 *   err_bound a-posteriori bound on |error of logP| from the arithmetic
 *   status    gbs_status of this pattern
 * Without a prior gbs_reserve covering the call, the call may synchronise once
 * to size its workspace. */
int gbs_prob(gbs_ctx *ctx, int M, const double *O, const double *logdet_sigmaQ,
             const uint64_t *patterns, int n_pat, int order, int precision, double *logP,
             double *kappa, double *err_bound, int32_t *status);

/* The whole path from HOST buffers: copies U, r and the patterns to the device,
 * builds the state, evaluates every pattern and copies the per-pattern results
 * back.  Synchronous.  Any of kappa_host, err_host, status_host may be NULL. */
int gbs_run_host(gbs_ctx *ctx, int M, const double *U_host, const double *r_host, double eta,
                 const uint64_t *patterns_host, int n_pat, int order, int precision,
                 double *logP_host, double *kappa_host, double *err_host, int32_t *status_host);

/* Whole-device click-number distribution (Methods, "Model": the sum of P(S) over the
 * C(M, n) patterns with n clicks; the paper's exact p(n) curve).  Every pattern S with n
 * clicks contains a subset Z in C(M - |Z|, n - |Z|) ways, so
 *   p(n) = det(sigma_Q)^{-1/2} sum_{z <= n} (-1)^{n - z} C(M - z, n - z) E_z,
 *   E_z  = sum over the subsets Z of the M modes with |Z| = z of det(A_Z)^{-1/2}:
 * one fixed-point sweep over all 2^M subsets with the terms binned by size (double-double
 * instead when a pivot leaves the fixed-point range: one readback decides), then the
 * binomial transform in double-double with exact binomials.  4 <= M <= 36 (2^M subsets:
 * 0.42 s at M = 30; the workspace holds 16 (M + 1) bytes per unit of 2^12..2^13 subsets,
 * 5..10 GB at M = 36).  Synchronises the stream once.  logp, kappa: M + 1 doubles (device; kappa may be NULL),
 * kappa[n] = sum_z C(M - z, n - z) E_z / |sum with signs|, the transform's cancellation;
 * logp[n] = NaN where the sum is not positive or a pivot was not.  Errors:
 * GBS_E_INVALID, GBS_E_CUDA, GBS_E_NOMEM. */
int gbs_click_distribution(gbs_ctx *ctx, int M, const double *O, const double *logdet_sigmaQ, double *logp,
                           double *kappa);

/* Photon-number sectors of the whole device's click-number distribution (Results,
 * "Calculation of sectors p_k(n)", and Methods, "Partition function": p(n) = sum_k p_k(n),
 * p_k(n) the probability of n clicks with k photons in the device).  With the sector
 * generating function of a set Z of modes, det(I - t O_Z)^{-1/2} (t marks each photon),
 *   G_n(t) = sum_k p_k(n) t^k = det(sigma_Q)^{-1/2} sum_{z <= n} (-1)^{n-z} C(M-z, n-z) E_z(t),
 *   E_z(t) = sum over the subsets Z with |Z| = z of det(I - t O_Z)^{-1/2},
 * evaluated at t_j = rho e^{2 pi i j / L}, j = 0..L/2, by a complex sweep over all 2^M
 * subsets binned by size (principal branch: I - t O_Z is accretive for |t| <= 1) in FP64
 * (precision GBS_FP64) or float-float (GBS_FF: ~48-bit parts on the FP32 pipes), then
 * p_k(n) = rho^-k / L sum_{j < L} G_n(t_j) e^{-2 pi i j k / L} (G_n(t_{L-j}) = conj G_n(t_j)).
 * 4 <= M <= 36; L a power of two in 4..4096 (sectors k >= L alias onto k mod L: choose L
 * beyond the photon numbers that matter); 0 < rho <= 1; 0 <= K < L.  even_only != 0 declares
 * that every odd sector vanishes (a lossless state: photons come in pairs, G_n(-t) = G_n(t)),
 * which halves the sweeps; the odd rows of pkn are then zero to rounding.  pkn: (K + 1) x
 * (M + 1) doubles (device), row k = p_k(0..M).  Cost: L/2 + 1 sweeps of 2^M subsets (L/4 + 1
 * with even_only).  Accuracy:
 * with FP64 subset terms each G_n(t_j) carries an absolute error of about 1e-16 (float-float:
 * ~1e-14) times the transform's cancellation (kappa of gbs_click_distribution) times p(n)
 * (|G_n(t)| <= p(n) for |t| <= 1), and p_k(n) that error times rho^-k.  NaN everywhere if
 * a pivot was zero.  Errors: GBS_E_INVALID, GBS_E_CUDA, GBS_E_NOMEM. */
int gbs_sector_distribution(gbs_ctx *ctx, int M, const double *O, const double *logdet_sigmaQ, int L, double rho,
                            int K, int even_only, int precision, double *pkn);

/* The approximation's fitted sector curves for one pattern S with n clicks (Results,
 * "Approximation scheme": p_k ~ exp(-f_j), and the paper's Fig. 3a): the same steps as
 * gbs_prob at order j (minors at the tilted contour points, DFT, per-sector factorial
 * moments, maximum-entropy fit of degree min(j, support - 1)), but each sector's whole
 * fitted distribution is returned, not only its all-clicked point: row k of curves
 * ((K + 1) x (n + 1) doubles, device) holds det(sigma_Q)^{-1/2} rho^-k q_k(v) at column
 * c = n - v, the estimate of P(c of the n detectors of S click, every other dark, k photons).
 * For S = all M modes this is the estimate of the whole device's sectors p_k(c)
 * (compare gbs_sector_distribution).  Sectors with fewer photons than clicks needed are
 * fitted too; rows past the pattern's sector range and sectors below the noise floor are
 * zero.  pattern: one device pattern; n must be its click count.  precision: GBS_FP64 or
 * GBS_FF.  logP, status: the pattern's estimate as gbs_prob (device, one each).  Errors:
 * GBS_E_INVALID (sizes, n not the pattern's clicks), GBS_E_CUDA, GBS_E_NOMEM. */
int gbs_approx_sector_curves(gbs_ctx *ctx, int M, const double *O, const double *logdet_sigmaQ,
                             const uint64_t *pattern, int n, int order, int precision, int K, double *curves,
                             double *logP, int32_t *status);

/* One batch split across GPUs (not in the paper; Methods, "Probability of any sample" is
 * the sum these slices partition).  The exact sum's work units -- (pattern, include /
 * exclude choice of the pattern's first modes), each 2^(s + 9) subsets in GBS_FX, 2^(s + 10)
 * or more in the other precisions once n is large enough -- are numbered over the batch
 * (patterns by decreasing n); slice `part` of `nparts` is the units
 * [U part / nparts, U (part + 1) / nparts) of the U in all, so equal unit counts give
 * equal work and a large pattern may be cut by its subset prefix.  gbs_prob_partial sweeps
 * one slice and writes, per pattern, the slice's partial sum as partial[3p..3p+2] =
 * (T_hi, T_lo, sum of |terms|) (zeros where the slice holds none of the pattern's units) and
 * pflag[p] (-1 invalid pattern; else bits 1 a pivot was not positive, 2 a pivot left the
 * fixed-point range, 4 the batch did not fit the reserved workspace).  Every rank runs it on
 * the same batch with its own part; the slices' outputs (24 + 4 bytes per pattern) are then
 * gathered in part order and gbs_prob_combine sums them per pattern in that order (TwoSum)
 * and returns what gbs_prob returns for the batch: logP, kappa, err_bound, status (outputs
 * may be NULL except logP).  partials: nparts x n_pat x 3 doubles, pflags: nparts x n_pat
 * int32, part-major (device).  precision: GBS_FX, GBS_DD, GBS_FP64 or GBS_FP32_SPLIT, the
 * same in both calls (GBS_FX patterns out of range come back GBS_E_RANGE: run them again
 * in GBS_DD).  gbs_prob_partial may synchronise and grow the workspace as gbs_prob does.
 * Errors: GBS_E_INVALID, GBS_E_CUDA, GBS_E_NOMEM. */
int gbs_prob_partial(gbs_ctx *ctx, int M, const double *O, const uint64_t *patterns, int n_pat, int precision,
                     int part, int nparts, double *partial, int32_t *pflag);
int gbs_prob_combine(gbs_ctx *ctx, const double *logdet_sigmaQ, const uint64_t *patterns, int n_pat, int precision,
                     int nparts, const double *partials, const int32_t *pflags, double *logP, double *kappa,
                     double *err_bound, int32_t *status);

/* Approximation (order > 0) with FP64 or float-float minors: patterns of at least n_min
 * clicks run on the CTA-pair kernel (a thread-block cluster of two CTAs holding half of the
 * packed 2n x 2n inverse each) instead of one CTA.  Patterns above 79 clicks always do (their
 * inverse exceeds one SM's shared memory); the default n_min is 80.  A lower n_min routes
 * smaller patterns through the pair kernel too (the results are the same up to rounding);
 * the tests use it to check that kernel against the oracle on small patterns.  Not in the
 * paper.  n_min in [3, 80], else GBS_E_INVALID. */
int gbs_set_pair_from(gbs_ctx *ctx, int n_min);

/* Allocation-free variant of gbs_prob for the exact sum (order 0).  The paper
 * has no counterpart: this serves callers that cannot call cudaMalloc (code
 * running under another owner's stream capture, processes whose device memory
 * is held by another framework's pool, serving loops that must not wait on the
 * allocator).  Its scratch is one fixed 8 MiB array in the library's device
 * memory (held by every GPU that loads the library until exit): at most 16384
 * patterns, and n_pat patterns of up to n_max clicks must fit in it, else the
 * call returns GBS_E_INVALID with a message.  Patterns with more than n_max
 * clicks may overflow it; then every pattern reports GBS_E_NOMEM.  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture.  All calls share the array:
 * calls that overlap on the GPU (other streams, other threads) race and must
 * be serialised by the caller.  precision: GBS_FX, GBS_DD, GBS_FP64 or GBS_FP32_SPLIT
 * (GBS_AUTO is not taken: its double-double rerun needs buffers of its own); a GBS_FX
 * pattern outside the fixed-point range reports GBS_E_RANGE and is not rerun, so
 * evaluate such patterns again with GBS_DD.  No allocation, no synchronisation. */
int gbs_prob_noalloc(gbs_ctx *ctx, int M, const double *O, const double *logdet_sigmaQ,
                     const uint64_t *patterns, int n_pat, int n_max, int precision, double *logP,
                     double *kappa, double *err_bound, int32_t *status);

/* ---- gradients (not in the paper) ---------------------------------------
 * L = sum_p w[p] log P(S_p) (exact probabilities, n <= 24 clicks per pattern).
 * With A = sigma_Q^{-1}, dT = tr(Gbar dA_S), Gbar = sum_Z (-1)^{n-|Z|} (-1/2)
 * det(A_Z)^{-1/2} A_Z^{-1} (the trace formula d det^{-1/2} = -1/2 det^{-1/2}
 * tr(A^{-1} dA)), i.e. Gbar = dT/dA_S, computed in double-double (Gbar and T
 * cancel alike) by reverse mode through the include/exclude Schur recursion that
 * evaluates T (O(2^n) work per pattern):
 *   dL/dsigma_Q = -1/2 (sum w) A - A H A,  H = sum_p (w_p / T_p) Gbar_p (embedded).
 * w: n_pat doubles (device).  dsigmaQ: 2M x 2M out (device).  logP, status:
 * optional per-pattern outputs (the double-double log P).  Synchronises once
 * (pattern sizes are checked on the host); GBS_E_INVALID for a pattern with
 * more than 24 clicks or a detector >= M. */
int gbs_grad(gbs_ctx *ctx, int M, const double *O, const double *logdet_sigmaQ,
             const uint64_t *patterns, int n_pat, const double *w, double *dsigmaQ, double *logP,
             int32_t *status);

/* Gradient of the order-j moment approximation (j = order, 1..4; FP64 minors), the
 * same L and output as gbs_grad: dL/dsigma_Q = -1/2 (sum w) A - A H A with
 * H = sum_p w_p dlog(sum_k part_k rho^-k)/dA_S (embedded), in reverse mode through the
 * approximation's steps (Methods, "Partition function", "Moments calculation",
 * "Approximation method"): the sum over sectors; the fit, by the implicit derivative
 * of its moment conditions at the solution (d part / d mu'_i = e^{-a_0} (Hn^-1)_0i,
 * Hn the fit's Newton matrix); the Stirling moments; the discrete Fourier transform;
 * and every group minor, through d Z_{S\W}(t)/dA_S = -1/2 t Z_{S\W}(t)
 * (G - G_{.W} G_WW^-1 G_{W.}), G = (I - t O_S)^-1.  The contour radius, the sector
 * range and the order each sector's fit used are those of the forward pass (held
 * fixed: log P is piecewise smooth in them).  Per pattern and contour point,
 * (j + j(j-1)/2) C(n, j) eliminations of at most 8 x 8 plus O(n^3).  w: n_pat doubles (device).  dsigmaQ: 2M x 2M out (device).  logP,
 * status: optional per-pattern outputs of the forward pass (as gbs_prob with
 * GBS_FP64; GBS_E_NOT_SPD also when the adjoint met a non-positive pivot).  A
 * pattern whose status is not GBS_OK or GBS_E_FIT adds nothing to H.  Synchronises
 * (pattern sizes are checked on the host); GBS_E_INVALID for a pattern with more
 * than 48 clicks or a detector >= M, or an order outside 1..4.  May grow the
 * context's buffers (see gbs_reserve). */
int gbs_grad_approx(gbs_ctx *ctx, int M, const double *O, const double *logdet_sigmaQ,
                    const uint64_t *patterns, int n_pat, int order, const double *w, double *dsigmaQ,
                    double *logP, int32_t *status);

/* Chain to the state parameters of gbs_build_state: from dL/dsigma_Q (= dL/dsigma)
 * to dU (M x M complex interleaved: dL/dRe U + i dL/dIm U), dr (M) and deta (one
 * double), all on the device. */
int gbs_grad_params(gbs_ctx *ctx, int M, const double *U, const double *r, double eta,
                    const double *dsigmaQ, double *dU, double *dr, double *deta);

/* Rectangular interferometer mesh (Clements et al., Optica 3, 1460 (2016)):
 * U = T_{last} ... T_1, cell c acts on modes (m_c, m_c + 1) as
 * [[e^{i phi} cos theta, -sin theta], [e^{i phi} sin theta, cos theta]]; layer
 * l = 0..M-1 holds the pairs whose first mode has the parity of l.  theta, phi:
 * M(M-1)/2 doubles each; U: M x M complex interleaved (device). */
int gbs_clements_unitary(gbs_ctx *ctx, int M, const double *theta, const double *phi, double *U);
/* Reverse pass through the mesh: dtheta, dphi from dU (same convention as
 * gbs_grad_params) and the mesh's U. */
int gbs_clements_grad(gbs_ctx *ctx, int M, const double *theta, const double *phi, const double *U,
                      const double *dU, double *dtheta, double *dphi);

/* ---- synthetic click patterns -------------------------------------------
 * Pattern i draws uint32 words w_0, w_1, ... from Philox4x32-10 (Salmon et al.,
 * SC'11) with key (seed mod 2^32, seed / 2^32) and counters (i, block, stream, 0);
 * n = n_lo + floor(w_0 (n_hi - n_lo + 1) / 2^32); then for k < n:
 * j = k + floor(w_{k+1} (M - k) / 2^32), swap perm[k], perm[j]; the clicked set is
 * perm[0..n-1].  out: n_pat x 2 uint64.  Bit-exact with the host generator. */
int gbs_gen_patterns(gbs_ctx *ctx, uint64_t seed, uint32_t stream, int M, int n_lo, int n_hi,
                     int n_pat, uint64_t *out);

/* ---- measurement helpers -------------------------------------------------
 * Kernel timing: while enabled, the context records a CUDA event pair on its
 * stream around every launch of the subset-sweep kernel.  gbs_timing_read
 * synchronises the stream and returns the summed device time (ms) and launch
 * count since the last reset (reset != 0 clears them).  At most 4096 launches
 * are kept between reads; older pairs are folded in as the ring wraps. */
int gbs_timing_enable(gbs_ctx *ctx, int enable);
int gbs_timing_read(gbs_ctx *ctx, int reset, double *sweep_ms, long long *sweep_launches);

/*
 * Peak arithmetic throughput of this GPU at the clocks of the run, in FLOP/s.
 * kind 0 / 1: the FP32 / FP64 FMA pipes from a register-resident dependent-FMA
 * loop (one FMA = 2 FLOP).  kind 2 / 3: the sweep's own fused Schur-update entry
 * (4 FLOP: c - w0 b0 - w1 b1 in double-double; c + t_i + t_j - (u'_i0 u'_j0 +
 * u'_i1 u'_j1) with two unsigned 128-bit products in fixed point), from a loop of
 * independent entries: the ceiling of the sweep in those precisions.  kind 4: 32-bit
 * integer multiply-adds per second (IMAD, eight independent chains per thread; one
 * per multiply-add, not 2), the issue rate of the pipe that carries the fixed-point
 * products.  Synchronous.  The scratch buffer it writes is the context's own. */
int gbs_peak_flops(gbs_ctx *ctx, int kind, double *flops);

#ifdef __cplusplus
}
#endif
#endif /* GBS_H */
