/*
 * oracle.c -- plain FP64 CPU oracle for click-pattern probabilities of a
 * Gaussian boson sampler with threshold detectors.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code, header or constant with the CUDA library, and it is deliberately
 * slow: every subset determinant is a fresh Cholesky factorisation.
 *
 * What it computes (paper sections cited by name):
 *  - Methods, "Model": squeezed inputs r_j, interferometer U (a_out = U a_in),
 *    extended here to uniform loss eta by the covariance form
 *        sigma   = eta R sigma_in R^T + (1 - eta) I/2,
 *        sigma_Q = sigma + I/2,  A = sigma_Q^{-1},  O = I - A,
 *    in xp order (x_1..x_M, p_1..p_M), hbar = 1, vacuum sigma = I/2.
 *  - Methods, "Probability of any sample" and Eq. (p(n)): the probability of a
 *    click pattern S is the signed sum over the sub-ensembles Z of S,
 *        P(S) = det(sigma_Q)^{-1/2} sum_{Z subset S} (-1)^{|S|-|Z|} det(A_Z)^{-1/2},
 *    one determinant per subset ("2^n determinants").  A_Z is the principal
 *    submatrix of A on the x and p rows of the modes in Z.
 *  - The signed sum is accumulated with the error-free Sum2 of Ogita, Rump and
 *    Oishi (SIAM J. Sci. Comput. 26, 2005) in subset-mask order 0..2^n-1.
 *  - For click patterns far below their expected click count the signed sum
 *    cancels by many orders of magnitude (kappa = sum|term| / |T| up to 1e13 and
 *    beyond), and FP64 subset determinants leave ~kappa * 1e-16 error.  The
 *    double-double variants (orc_subset_sum_dd*) compute every Cholesky and
 *    the sum with ~106-bit arithmetic.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_NOT_SPD 5
#define ORC_INVALID 1

/* Cholesky a = L L^T in place (lower triangle, row-major n x n).  Returns 0 or
 * ORC_NOT_SPD if a pivot is not positive. */
static int cholesky(double *a, int n) {
    for (int j = 0; j < n; ++j) {
        double d = a[j * n + j];
        for (int k = 0; k < j; ++k) d -= a[j * n + k] * a[j * n + k];
        if (!(d > 0.0)) return ORC_NOT_SPD;
        d = sqrt(d);
        a[j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double s = a[i * n + j];
            for (int k = 0; k < j; ++k) s -= a[i * n + k] * a[j * n + k];
            a[i * n + j] = s / d;
        }
    }
    return ORC_OK;
}

/* Error-free transformation a + b = s + e. */
static void two_sum(double a, double b, double *s, double *e) {
    double x = a + b;
    double bp = x - a;
    *e = (a - (x - bp)) + (b - bp);
    *s = x;
}

/*
 * State build.  U: M*M complex row-major, interleaved (re, im).  r: M squeezing
 * parameters (0 = vacuum input).  Outputs (may be NULL): sigma, sigmaQ, A, O,
 * each 2M x 2M row-major in xp order; logdet_sigmaQ.  Returns 0 or error code.
 */
int orc_build_state(int M, const double *U, const double *r, double eta, double *sigma,
                    double *sigmaQ, double *A, double *O, double *logdet_sigmaQ) {
    if (M <= 0 || !(eta > 0.0) || eta > 1.0) return ORC_INVALID;
    int N = 2 * M;
    double *R = calloc((size_t)N * N, sizeof(double));
    double *S = calloc((size_t)N * N, sizeof(double));
    double *L = calloc((size_t)N * N, sizeof(double));
    if (!R || !S || !L) { free(R); free(S); free(L); return ORC_INVALID; }
    /* R = [[Re U, -Im U], [Im U, Re U]]: x_out = Re U x - Im U p, p_out = Im U x + Re U p. */
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) {
            double re = U[2 * (i * M + j)], im = U[2 * (i * M + j) + 1];
            R[i * N + j] = re;
            R[i * N + (j + M)] = -im;
            R[(i + M) * N + j] = im;
            R[(i + M) * N + (j + M)] = re;
        }
    /* sigma_in = diag(e^{-2r}/2 (x), e^{2r}/2 (p)); sigma = eta R sigma_in R^T + (1-eta)/2 I. */
    for (int i = 0; i < N; ++i)
        for (int k = 0; k < N; ++k) {
            double s = 0.0;
            for (int j = 0; j < M; ++j) {
                s += R[i * N + j] * R[k * N + j] * 0.5 * exp(-2.0 * r[j]);
                s += R[i * N + j + M] * R[k * N + j + M] * 0.5 * exp(2.0 * r[j]);
            }
            S[i * N + k] = eta * s + (i == k ? 0.5 * (1.0 - eta) : 0.0);
        }
    if (sigma) memcpy(sigma, S, sizeof(double) * N * N);
    for (int i = 0; i < N; ++i) S[i * N + i] += 0.5; /* sigma_Q */
    if (sigmaQ) memcpy(sigmaQ, S, sizeof(double) * N * N);
    memcpy(L, S, sizeof(double) * N * N);
    int st = cholesky(L, N);
    if (st) { free(R); free(S); free(L); return st; }
    double ld = 0.0;
    for (int i = 0; i < N; ++i) ld += 2.0 * log(L[i * N + i]);
    if (logdet_sigmaQ) *logdet_sigmaQ = ld;
    /* A = sigma_Q^{-1}: solve L L^T x = e_c for every column c. */
    double *col = R; /* reuse */
    for (int c = 0; c < N; ++c) {
        for (int i = 0; i < N; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) s -= L[i * N + k] * col[k];
            col[i] = s / L[i * N + i];
        }
        for (int i = N - 1; i >= 0; --i) {
            double s = col[i];
            for (int k = i + 1; k < N; ++k) s -= L[k * N + i] * col[k];
            col[i] = s / L[i * N + i];
        }
        for (int i = 0; i < N; ++i) {
            if (A) A[i * N + c] = col[i];
            if (O) O[i * N + c] = (i == c ? 1.0 : 0.0) - col[i];
        }
    }
    free(R); free(S); free(L);
    return ORC_OK;
}

/*
 * Signed subset sum over the masks [z_begin, z_end) of the n modes `modes`:
 *   out[0] + out[1] = sum_z (-1)^{n-|Z|} det(A_Z)^{-1/2}  (Sum2, hi + lo)
 *   out[2]          = sum_z det(A_Z)^{-1/2}
 * A is the 2M x 2M matrix (I - O).  Returns 0 or ORC_NOT_SPD.
 */
int orc_subset_sum(int M, const double *A, const int *modes, int n, uint64_t z_begin,
                   uint64_t z_end, double *out) {
    int N = 2 * M;
    double *B = malloc(sizeof(double) * 4 * (size_t)n * n + 1);
    int *idx = malloc(sizeof(int) * 2 * (size_t)n + 1);
    if (!B || !idx) { free(B); free(idx); return ORC_INVALID; }
    double s = 0.0, c = 0.0, sabs = 0.0;
    int status = ORC_OK;
    for (uint64_t z = z_begin; z < z_end; ++z) {
        int k = 0;
        for (int a = 0; a < n; ++a)
            if (z >> a & 1) { idx[2 * k] = modes[a]; idx[2 * k + 1] = modes[a] + M; ++k; }
        int d = 2 * k;
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) B[i * d + j] = A[idx[i] * N + idx[j]];
        double tau = 1.0;
        if (d) {
            if (cholesky(B, d)) { status = ORC_NOT_SPD; break; }
            for (int i = 0; i < d; ++i) tau /= B[i * d + i];
        }
        double term = ((n - k) & 1) ? -tau : tau;
        double e;
        two_sum(s, term, &s, &e);
        c += e;
        sabs += tau;
    }
    out[0] = s; out[1] = c; out[2] = sabs;
    free(B); free(idx);
    return status;
}

/* ---- double-double arithmetic (Dekker 1971; Hida, Li & Bailey 2001) -------
 * A value is hi + lo with |lo| <= ulp(hi)/2; about 106 significant bits.  Used
 * for subset determinants whose signed sum cancels beyond FP64 precision. */
typedef struct {
    double hi, lo;
} dd;

static dd dd_two_sum(double a, double b) {
    dd r;
    two_sum(a, b, &r.hi, &r.lo);
    return r;
}
static dd dd_quick(double a, double b) { /* requires |a| >= |b| */
    dd r;
    r.hi = a + b;
    r.lo = b - (r.hi - a);
    return r;
}
static dd dd_two_prod(double a, double b) {
    dd r;
    r.hi = a * b;
    r.lo = fma(a, b, -r.hi);
    return r;
}
static dd dd_add(dd a, dd b) {
    dd s = dd_two_sum(a.hi, b.hi), t = dd_two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = dd_quick(s.hi, s.lo);
    s.lo += t.lo;
    return dd_quick(s.hi, s.lo);
}
static dd dd_neg(dd a) {
    dd r = {-a.hi, -a.lo};
    return r;
}
static dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
static dd dd_mul(dd a, dd b) {
    dd p = dd_two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return dd_quick(p.hi, p.lo);
}
static dd dd_div(dd a, dd b) {
    double q1 = a.hi / b.hi;
    dd r = dd_sub(a, dd_mul((dd){q1, 0.0}, b));
    double q2 = r.hi / b.hi;
    r = dd_sub(r, dd_mul((dd){q2, 0.0}, b));
    double q3 = r.hi / b.hi;
    return dd_add(dd_quick(q1, q2), (dd){q3, 0.0});
}
static dd dd_sqrt(dd a) { /* one Newton step from the double square root */
    double x = sqrt(a.hi);
    dd r = dd_sub(a, dd_two_prod(x, x));
    return dd_two_sum(x, r.hi / (2.0 * x));
}

/* cholesky() in double-double; a holds n*n dd values (lower triangle used). */
static int cholesky_dd(dd *a, int n) {
    for (int j = 0; j < n; ++j) {
        dd d = a[j * n + j];
        for (int k = 0; k < j; ++k) d = dd_sub(d, dd_mul(a[j * n + k], a[j * n + k]));
        if (!(d.hi > 0.0)) return ORC_NOT_SPD;
        d = dd_sqrt(d);
        a[j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            dd s = a[i * n + j];
            for (int k = 0; k < j; ++k) s = dd_sub(s, dd_mul(a[i * n + k], a[j * n + k]));
            a[i * n + j] = dd_div(s, d);
        }
    }
    return ORC_OK;
}

/*
 * orc_subset_sum in double-double: every subset Cholesky and the signed sum
 * carry ~106 bits, so the result keeps its accuracy when the sum cancels by
 * many orders of magnitude.  A is the FP64 matrix (I - O) (exact inputs).
 * out: (hi, lo) of T and sum_Z det(A_Z)^{-1/2}.
 */
int orc_subset_sum_dd(int M, const double *A, const int *modes, int n, uint64_t z_begin,
                      uint64_t z_end, double *out) {
    int N = 2 * M;
    dd *B = malloc(sizeof(dd) * 4 * (size_t)n * n + 1);
    int *idx = malloc(sizeof(int) * 2 * (size_t)n + 1);
    if (!B || !idx) { free(B); free(idx); return ORC_INVALID; }
    dd sum = {0.0, 0.0};
    double sabs = 0.0;
    int status = ORC_OK;
    for (uint64_t z = z_begin; z < z_end; ++z) {
        int k = 0;
        for (int a = 0; a < n; ++a)
            if (z >> a & 1) { idx[2 * k] = modes[a]; idx[2 * k + 1] = modes[a] + M; ++k; }
        int d = 2 * k;
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) B[i * d + j] = (dd){A[idx[i] * N + idx[j]], 0.0};
        dd tau = {1.0, 0.0};
        if (d) {
            if (cholesky_dd(B, d)) { status = ORC_NOT_SPD; break; }
            for (int i = 0; i < d; ++i) tau = dd_div(tau, B[i * d + i]);
        }
        sum = ((n - k) & 1) ? dd_sub(sum, tau) : dd_add(sum, tau);
        sabs += tau.hi;
    }
    out[0] = sum.hi; out[1] = sum.lo; out[2] = sabs;
    free(B); free(idx);
    return status;
}

/* orc_subset_sum_dd split into mask ranges run in parallel, merged in order. */
int orc_subset_sum_dd_parallel(int M, const double *A, const int *modes, int n, int nchunk,
                               int nthreads, double *out) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    uint64_t total = (uint64_t)1 << n;
    if (nchunk < 1) nchunk = 1;
    double *part = calloc((size_t)nchunk * 3, sizeof(double));
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int c = 0; c < nchunk; ++c) {
        uint64_t b = total * (uint64_t)c / (uint64_t)nchunk;
        uint64_t e = total * (uint64_t)(c + 1) / (uint64_t)nchunk;
        bad |= orc_subset_sum_dd(M, A, modes, n, b, e, part + 3 * c);
    }
    dd sum = {0.0, 0.0};
    double sabs = 0.0;
    for (int c = 0; c < nchunk; ++c) {
        sum = dd_add(sum, (dd){part[3 * c], part[3 * c + 1]});
        sabs += part[3 * c + 2];
    }
    out[0] = sum.hi; out[1] = sum.lo; out[2] = sabs;
    free(part);
    return bad ? ORC_NOT_SPD : ORC_OK;
}

/*
 * Adjoint of the signed subset sum (the gradient path; not in the paper): with
 * d det(A_Z)^{-1/2} = -1/2 det(A_Z)^{-1/2} tr(A_Z^{-1} dA_Z),
 *     dT = tr(Gbar dA_S),  Gbar = sum_Z (-1)^{n-|Z|} (-1/2) tau_Z embed(A_Z^{-1}).
 * Every subset Cholesky, inverse and the sums are double-double.  Rows of the
 * 2n x 2n Gbar are (x, p) pairs of the modes of S in order: row 2a + alpha.
 * Outputs: Gbar as hi and lo arrays (2n x 2n each), T as (hi, lo).
 */
int orc_grad_subsets_dd(int M, const double *A, const int *modes, int n, double *g_hi,
                        double *g_lo, double *T) {
    int N = 2 * M, D = 2 * n;
    dd *G = calloc((size_t)D * D + 1, sizeof(dd));
    dd *B = malloc(sizeof(dd) * (size_t)D * D + 1);
    dd *Li = malloc(sizeof(dd) * (size_t)D * D + 1);
    int *idx = malloc(sizeof(int) * (size_t)D + 1), *loc = malloc(sizeof(int) * (size_t)D + 1);
    if (!G || !B || !Li || !idx || !loc) { free(G); free(B); free(Li); free(idx); free(loc); return ORC_INVALID; }
    dd sum = {0.0, 0.0};
    int status = ORC_OK;
    for (uint64_t z = 0; z < ((uint64_t)1 << n); ++z) {
        int k = 0;
        for (int a = 0; a < n; ++a)
            if (z >> a & 1) {
                idx[2 * k] = modes[a]; idx[2 * k + 1] = modes[a] + M;
                loc[2 * k] = 2 * a; loc[2 * k + 1] = 2 * a + 1;
                ++k;
            }
        int d = 2 * k;
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) B[i * d + j] = (dd){A[idx[i] * N + idx[j]], 0.0};
        dd tau = {1.0, 0.0};
        if (d) {
            if (cholesky_dd(B, d)) { status = ORC_NOT_SPD; break; }
            for (int i = 0; i < d; ++i) tau = dd_div(tau, B[i * d + i]);
            /* Li = L^{-1} (lower triangular) */
            for (int c = 0; c < d; ++c) {
                for (int i = 0; i < c; ++i) Li[i * d + c] = (dd){0.0, 0.0};
                Li[c * d + c] = dd_div((dd){1.0, 0.0}, B[c * d + c]);
                for (int i = c + 1; i < d; ++i) {
                    dd s2 = {0.0, 0.0};
                    for (int m = c; m < i; ++m) s2 = dd_add(s2, dd_mul(B[i * d + m], Li[m * d + c]));
                    Li[i * d + c] = dd_neg(dd_div(s2, B[i * d + i]));
                }
            }
            /* (A_Z^{-1})_{ij} = sum_m Li_mi Li_mj, weighted into Gbar */
            dd c0 = dd_mul(tau, (dd){((n - k) & 1) ? 0.5 : -0.5, 0.0});
            for (int i = 0; i < d; ++i)
                for (int j = 0; j < d; ++j) {
                    dd s2 = {0.0, 0.0};
                    int m0 = i > j ? i : j;
                    for (int m = m0; m < d; ++m) s2 = dd_add(s2, dd_mul(Li[m * d + i], Li[m * d + j]));
                    dd *gp = &G[loc[i] * D + loc[j]];
                    *gp = dd_add(*gp, dd_mul(c0, s2));
                }
        }
        sum = ((n - k) & 1) ? dd_sub(sum, tau) : dd_add(sum, tau);
    }
    for (int i = 0; i < D * D; ++i) { g_hi[i] = G[i].hi; g_lo[i] = G[i].lo; }
    T[0] = sum.hi; T[1] = sum.lo;
    free(G); free(B); free(Li); free(idx); free(loc);
    return status;
}

static int pattern_modes(uint64_t lo, uint64_t hi, int M, int *modes) {
    int n = 0;
    for (int i = 0; i < M; ++i) {
        uint64_t w = i < 64 ? lo : hi;
        if (w >> (i & 63) & 1) modes[n++] = i;
    }
    return n;
}

/*
 * Exact log-probability of n_pat click patterns (pairs of uint64 words).
 *   logP[p]  = -logdet_sigmaQ/2 + log T_p
 *   T[2p..]  = T_p as (hi, lo);  sumabs[p] = sum_Z det(A_Z)^{-1/2}
 *   status[p] = 0, ORC_NOT_SPD, or 4 if T_p <= 0.
 * OpenMP over patterns (nthreads <= 0: library default).  n <= 40.
 */
int orc_prob_exact(int M, const double *A, double logdet_sigmaQ, const uint64_t *patterns,
                   int n_pat, double *logP, double *T, double *sumabs, int *status,
                   int nthreads, int use_dd) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int p = 0; p < n_pat; ++p) {
        int modes[128];
        int n = pattern_modes(patterns[2 * p], patterns[2 * p + 1], M, modes);
        double out[3] = {0, 0, 0};
        int st = (n > 40) ? ORC_INVALID
                 : use_dd ? orc_subset_sum_dd(M, A, modes, n, 0, (uint64_t)1 << n, out)
                          : orc_subset_sum(M, A, modes, n, 0, (uint64_t)1 << n, out);
        double t = out[0] + out[1];
        if (!st && !(t > 0.0)) st = 4;
        status[p] = st;
        bad |= st != 0;
        T[2 * p] = out[0];
        T[2 * p + 1] = out[1];
        sumabs[p] = out[2];
        /* log(hi + lo) = log(hi) + log1p(lo / hi) keeps the double-double digits */
        logP[p] = st ? NAN : -0.5 * logdet_sigmaQ + log(out[0]) + log1p(out[1] / out[0]);
    }
    return bad ? 4 : ORC_OK;
}

/*
 * One large pattern split into `nchunk` mask ranges run in parallel, merged in
 * range order with Sum2.  out: (hi, lo, sumabs).
 */
int orc_subset_sum_parallel(int M, const double *A, const int *modes, int n, int nchunk,
                            int nthreads, double *out) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    uint64_t total = (uint64_t)1 << n;
    if (nchunk < 1) nchunk = 1;
    double *part = calloc((size_t)nchunk * 3, sizeof(double));
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int c = 0; c < nchunk; ++c) {
        uint64_t b = total * (uint64_t)c / (uint64_t)nchunk;
        uint64_t e = total * (uint64_t)(c + 1) / (uint64_t)nchunk;
        bad |= orc_subset_sum(M, A, modes, n, b, e, part + 3 * c);
    }
    double s = 0.0, cc = 0.0, sabs = 0.0;
    for (int c = 0; c < nchunk; ++c) {
        double e;
        two_sum(s, part[3 * c], &s, &e);
        cc += e + part[3 * c + 1];
        sabs += part[3 * c + 2];
    }
    out[0] = s; out[1] = cc; out[2] = sabs;
    free(part);
    return bad ? ORC_NOT_SPD : ORC_OK;
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
