// The paper's moment approximation (Methods, "Partition function", "Moments
// calculation", "Approximation method") for click patterns S of n detectors:
//
//  1. sectors: Z_Z(t) = det(I - t O_Z)^{-1/2} = sum_k c_k[Z] t^k, where
//     c_k[Z] det(sigma_Q)^{-1/2} = P(k photons in Z, vacuum elsewhere).  The
//     coefficients are extracted by a discrete Fourier transform over
//     t_l = e^{i nu_l}, nu_l = 2 pi l / L (the paper's sum over nu);
//  2. moments: the minors with w <= j detectors removed give the factorial
//     moments of the vacuum count v in every sector,
//        D_w(t) = sum_{|W| = w} Z_{S \ W}(t),  D_w^(k) = sum_v C(v, w) q_k(v);
//     by Jacobi's identity Z_{S \ W}(t) = Z_S(t) det(G_WW)^{-1/2}, G = (I - t O_S)^{-1};
//  3. inverse moment problem: q_k(v) ~ exp(-f(v)), deg f <= j, moments 0..j
//     matched (convex maximum-entropy dual, damped Newton);
//  4. P(S) ~ det(sigma_Q)^{-1/2} sum_k exp(-f_k(0)).
//
// The circle |t| = rho is tilted to the Chernoff saddle of sector n so that the
// sectors carrying the all-clicked point (far in the upper tail for improbable
// patterns) sit near the peak of c_k rho^k and keep their relative precision.
// Kernels: approx_plan (per pattern: rho, and a rigorous bound K on the sector
// index with tilted tail < 1e-14 Z_S(rho) from Chernoff's inequality; DFT length
// L = K + 1), approx_minors (one CTA per (pattern, nu_l), l <= L/2 by conjugate
// symmetry), approx_fit (one CTA per pattern: inverse DFT, fits, sum).
#include <cooperative_groups.h>
#include <type_traits>
#include <math.h>

#include "ff.cuh"
#include "gbs_internal.cuh"

namespace cg = cooperative_groups;

#ifndef GBS_FF_FMS_INLINE
#define GBS_FF_FMS_INLINE __noinline__
#endif

namespace {

constexpr int kMaxOrder = 4;
constexpr int kMinorThreads = 256;
constexpr int kDftThreads = 128;
constexpr int kSecThreads = 256;   // one warp per sector
constexpr int kSumThreads = 128;   // one warp per pattern
constexpr int kPlanThreads = 256;
constexpr double kTailEps = 1e-14;
constexpr double kFlagShare = 1e-4;     // fallback reported when such sectors carry this share of P
constexpr int kNumRho = 15;
__constant__ double kRhos[kNumRho] = {1.0, 1.02, 1.05, 1.1, 1.15, 1.2, 1.25, 1.3, 1.4, 1.5, 1.7, 2.0, 2.5, 3.0, 4.0};
constexpr int kMaxK = 4095;
constexpr int kApproxMaxN = 112;

__host__ __device__ constexpr int sym(int d) { return d * (d + 1) / 2; }
__host__ __device__ constexpr int pidx(int d, int i, int j) { return i * d - (i * (i - 1)) / 2 + (j - i); }
__device__ __forceinline__ int pidx_any(int d, int i, int j) { return i <= j ? pidx(d, i, j) : pidx(d, j, i); }

// ---- complex arithmetic ---------------------------------------------------------
template <typename R> struct cx {
    R re, im;
};
template <typename R> __device__ __forceinline__ cx<R> mk(R a, R b) { return cx<R>{a, b}; }
template <typename R> __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R> __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R> __device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R> __device__ __forceinline__ cx<R> cinv(cx<R> a) {
    const R d = R(1) / (a.re * a.re + a.im * a.im);
    return {a.re * d, -a.im * d};
}
__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_r(double x) { return rsqrt(x); }
__device__ __forceinline__ ff rsqrt_r(ff x) { return ff_rsqrt(x); }
// principal p^{-1/2} for Re p > 0: with a = |p| and s = sqrt((a + Re p)/2) (no
// cancellation: Re p > 0), sqrt(p) = s + i Im p / (2 s) and p^{-1/2} = (s - i Im p/(2 s)) / a;
// two reciprocal square roots, no division
template <typename R> __device__ __forceinline__ cx<R> crsqrt(cx<R> p) {
    const R n2 = p.re * p.re + p.im * p.im;
    const R ra = rsqrt_r(n2);
    const R h = (n2 * ra + p.re) * R(0.5);
    const R rh = rsqrt_r(h);
    return {h * rh * ra, -p.im * ra * rh * R(0.5)};
}
// float-float complex products, reciprocals and roots as shared (non-inlined) calls (the
// overloads win over the templates): inlined everywhere they overflowed the instruction
// cache (-33% time on the order-4 minors with these three out of line)
static __device__ __noinline__ cx<ff> operator*(cx<ff> a, cx<ff> b) {
    return {ff_dot2(a.re, b.re, -a.im, b.im), ff_dot2(a.re, b.im, a.im, b.re)};
}
// e - a b: one fused form per part for float-float (see ff_fms2)
template <typename R> __device__ __forceinline__ cx<R> cfms(cx<R> e, cx<R> a, cx<R> b) { return e - a * b; }
__device__ __forceinline__ cx<ff> cfms_ff(cx<ff> e, cx<ff> a, cx<ff> b) {
    return {ff_fms2(e.re, a.re, b.re, -a.im, b.im), ff_fms2(e.im, a.re, b.im, a.im, b.re)};
}
// out of line in the group terms (their unrolled loops hold dozens of these: inlined, the
// code overflows the instruction cache); inline in the inverse's one-line update loop
static __device__ GBS_FF_FMS_INLINE cx<ff> cfms(cx<ff> e, cx<ff> a, cx<ff> b) { return cfms_ff(e, a, b); }
template <typename R> __device__ __forceinline__ cx<R> cfms_inl(cx<R> e, cx<R> a, cx<R> b) { return e - a * b; }
__device__ __forceinline__ cx<ff> cfms_inl(cx<ff> e, cx<ff> a, cx<ff> b) { return cfms_ff(e, a, b); }
static __device__ __noinline__ cx<ff> cinv(cx<ff> a) { return cinv<ff>(a); }
static __device__ __noinline__ cx<ff> crsqrt(cx<ff> p) { return crsqrt<ff>(p); }
__device__ __forceinline__ cx<double> widen(cx<float> a) { return {(double)a.re, (double)a.im}; }

// ---- the four-detector step of the pair phases ----------------------------------------
// K entry: v - sum_k x_k y_k over the four rows of the pair's Schur factor (x = w_c, y = w_d)
template <typename R>
__device__ __forceinline__ cx<R> rank4_entry(cx<R> v, const cx<R> *x, const cx<R> *y, int i, int j) {
#pragma unroll
    for (int k = 0; k < 4; ++k) v = cfms(v, x[2 * k + i], y[2 * k + j]);
    return v;
}
// the term det(G_{P+c+d})^{-1/2} = f3_c det(S)^{-1/2}, S = H_d - K^T H_c^{-1} K, from K and the
// stored items of c (ic) and d (jd); *bad: a pivot of S not accretive
template <typename R> struct QuadTerm {
    cx<R> term;
    int bad;
};
template <typename R>
__device__ __forceinline__ QuadTerm<R> quad_term(cx<R> k00, cx<R> k01, cx<R> k10, cx<R> k11, const cx<R> *ic,
                                                 const cx<R> *jd) {
    const cx<R> K[2][2] = {{k00, k01}, {k10, k11}};
    const cx<R> i00 = ic[11], i01 = ic[12], i11 = ic[13];
    cx<R> X[2][2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        X[0][j] = i00 * K[0][j] + i01 * K[1][j];
        X[1][j] = i01 * K[0][j] + i11 * K[1][j];
    }
    const cx<R> s00 = cfms(cfms(jd[8], K[0][0], X[0][0]), K[1][0], X[1][0]);
    const cx<R> s01 = cfms(cfms(jd[9], K[0][0], X[0][1]), K[1][0], X[1][1]);
    const cx<R> s11 = cfms(cfms(jd[10], K[0][1], X[0][1]), K[1][1], X[1][1]);
    const cx<R> det = cfms(s00 * s11, s01, s01);
    QuadTerm<R> q;
    q.bad = !(s00.re > R(0)) || !(det.re * s00.re + det.im * s00.im > R(0));
    q.term = ic[14] * crsqrt(det);
    return q;
}
// float-float: each of these as one out-of-line call whose arithmetic is inline (the same
// operations as the shared complex calls, a few calls per four-detector group instead of
// ~30: their argument traffic cost more than the code they share)
__device__ __forceinline__ cx<ff> cmul_ff(cx<ff> a, cx<ff> b) {
    return {ff_dot2(a.re, b.re, -a.im, b.im), ff_dot2(a.re, b.im, a.im, b.re)};
}
static __device__ __noinline__ cx<ff> rank4_entry(cx<ff> v, const cx<ff> *x, const cx<ff> *y, int i, int j) {
#pragma unroll
    for (int k = 0; k < 4; ++k) v = cfms_ff(v, x[2 * k + i], y[2 * k + j]);
    return v;
}
static __device__ __noinline__ QuadTerm<ff> quad_term(cx<ff> k00, cx<ff> k01, cx<ff> k10, cx<ff> k11,
                                                      const cx<ff> *ic, const cx<ff> *jd) {
    const cx<ff> K[2][2] = {{k00, k01}, {k10, k11}};
    const cx<ff> i00 = ic[11], i01 = ic[12], i11 = ic[13];
    cx<ff> X[2][2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        X[0][j] = cmul_ff(i00, K[0][j]) + cmul_ff(i01, K[1][j]);
        X[1][j] = cmul_ff(i01, K[0][j]) + cmul_ff(i11, K[1][j]);
    }
    const cx<ff> s00 = cfms_ff(cfms_ff(jd[8], K[0][0], X[0][0]), K[1][0], X[1][0]);
    const cx<ff> s01 = cfms_ff(cfms_ff(jd[9], K[0][0], X[0][1]), K[1][0], X[1][1]);
    const cx<ff> s11 = cfms_ff(cfms_ff(jd[10], K[0][1], X[0][1]), K[1][1], X[1][1]);
    const cx<ff> det = cfms_ff(cmul_ff(s00, s11), s01, s01);
    QuadTerm<ff> q;
    q.bad = !(s00.re > ff(0.0f, 0.0f)) || !(det.re * s00.re + det.im * s00.im > ff(0.0f, 0.0f));
    q.term = cmul_ff(ic[14], crsqrt<ff>(det));
    return q;
}
__device__ __forceinline__ cx<double> widen(cx<double> a) { return a; }
__device__ __forceinline__ cx<double> widen(cx<ff> a) { return {ff_to_double(a.re), ff_to_double(a.im)}; }

// an entry of I - t O_S, t = cs + i sn, from the FP64 products (forming it in FP32 was
// measured no faster and raised the FP32 path's fit fallbacks)
template <typename R> __device__ __forceinline__ cx<R> init_entry(bool diag, double cs, double sn, double o) {
    return mk<R>(R((diag ? 1.0 : 0.0) - cs * o), R(-sn * o));
}

// per precision of the minors: largest pattern (the packed inverse must fit in shared
// memory) and the tilted-sector share below which a sector counts as rounding noise
template <typename R> struct MinorPrec;
template <> struct MinorPrec<double> {
    static constexpr int min_blocks = 1;
    static constexpr int nmax = 79;
    static constexpr bool pair = true;  // n in (nmax, 112] on a CTA pair
    static constexpr double sector_eps = 1e-12;
    static constexpr bool floor_flag = false;  // below the floor: the oracle's own reading of negligible sectors
};
template <> struct MinorPrec<ff> {
    // two CTAs per SM: capped at 128 registers (a few spills) it runs 14% faster than one
    // CTA of 255-register threads
    static constexpr int min_blocks = 2;
    static constexpr int nmax = 79;
    static constexpr bool pair = true;
    static constexpr double sector_eps = 1e-12;
    static constexpr bool floor_flag = false;
};
template <> struct MinorPrec<float> {
    static constexpr int min_blocks = 2;  // 127 registers: two CTAs per SM
    static constexpr int nmax = 112;
    static constexpr bool pair = false;
    static constexpr double sector_eps = 1e-6;  // moments resolved to ~1e-7 K
    static constexpr bool floor_flag = true;    // below it: unresolved, reported (GBS_E_FLOOR)
};

// ---- plan: sector bound and DFT length per pattern ---------------------------------
struct ApproxPlan {
    int *pat_n;           // clicks (-1 invalid)
    int *pat_L;           // DFT length
    double *pat_rho;      // contour radius
    long long *unit_off;  // n_pat + 1: units (pattern, l) with l = 0..L/2
    long long *total;     // total units (0 if over capacity)
    int *overflow;
    double *unit_D;       // 2 (j + 1) doubles per unit: D_w(t_l), w = 0..j
    int *unit_flag;       // per pattern: non-positive pivot seen
    long long *info;      // units, largest n, largest L, sectors (read back to size the launches)
    long long *sec_off;   // n_pat + 1: sectors k = 0..L-1 of each pattern
    double *pat_max;      // per pattern: largest tilted sector
    double *sec_D;        // (kMaxOrder + 1) per sector: D_w^(k), w = 0..order
    double *sec_part;     // per sector: fitted last point (negative: the fit fell back)
};

// log det(I - rho O_S) by Cholesky in shared memory (packed); +inf if not positive definite
__device__ double logdet_shift(const double *__restrict__ O, int M, const int *modes, int n, double rho,
                               double *S, double *s_red) {
    const int N = 2 * n, N2 = 2 * M, t = threadIdx.x;
    for (int f = t; f < N * N; f += blockDim.x) {
        int i = f / N, j = f - i * N;
        if (j < i) continue;
        int si = modes[i >> 1] + (i & 1) * M, sj = modes[j >> 1] + (j & 1) * M;
        S[pidx(N, i, j)] = (i == j ? 1.0 : 0.0) - rho * O[(size_t)si * N2 + sj];
    }
    __syncthreads();
    __shared__ int bad;
    __shared__ double ld;
    if (t == 0) { bad = 0; ld = 0.0; }
    __syncthreads();
    for (int k = 0; k < N; ++k) {
        double d = S[pidx(N, k, k)];
        if (!(d > 0.0)) { if (t == 0) bad = 1; }
        __syncthreads();
        if (bad) break;
        double inv = 1.0 / d;
        if (t == 0) ld += log(d);
        const int Dt = N - k - 1;
        for (int f = t; f < Dt * Dt; f += blockDim.x) {
            int i = k + 1 + f / Dt, j = k + 1 + f % Dt;
            if (j < i) continue;
            S[pidx(N, i, j)] -= S[pidx(N, k, i)] * S[pidx(N, k, j)] * inv;
        }
        __syncthreads();
    }
    (void)s_red;
    double r = bad ? INFINITY : ld;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kPlanThreads) approx_plan_kernel(int M, const double *__restrict__ O,
                                                                 const uint64_t *__restrict__ pats,
                                                                 int n_pat, int order, int n_limit,
                                                                 ApproxPlan pl) {
    extern __shared__ double smem_d[];
    __shared__ int modes[128];
    __shared__ int s_n;
    const int p = blockIdx.x, t = threadIdx.x;
    const uint64_t lo = pats[2 * p], hi = pats[2 * p + 1];
    if (t == 0) {
        int n = 0;
        bool ok = true;
        for (int i = 0; i < 128; ++i) {
            uint64_t w = i < 64 ? lo : hi;
            if (w >> (i & 63) & 1ull) {
                if (i >= M) ok = false;
                else modes[n++] = i;
            }
        }
        s_n = (ok && n <= n_limit) ? n : -1;
    }
    __syncthreads();
    const int n = s_n;
    int L = 1;
    double rho_t = 1.0;
    if (n > 0) {
        // log Z_S(rho) = -1/2 log det(I - rho O_S) on the radii where I -+ rho O_S are
        // positive definite (then I - t O_S is accretive on the whole circle |t| = rho)
        double lz[kNumRho];
        int nv = 0;
        for (int q = 0; q < kNumRho; ++q) {
            double lm = logdet_shift(O, M, modes, n, kRhos[q], smem_d, nullptr);
            if (!isfinite(lm)) break;
            if (q > 0 && !isfinite(logdet_shift(O, M, modes, n, -kRhos[q], smem_d, nullptr))) break;
            lz[q] = -0.5 * lm;
            nv = q + 1;
        }
        // contour radius: Chernoff saddle for sector n, argmin log Z(rho) - n log rho
        const int nc = nv > 1 ? nv - 1 : 1;
        int qt = 0;
        for (int q = 1; q < nc; ++q)
            if (lz[q] - n * log(kRhos[q]) < lz[qt] - n * log(kRhos[qt])) qt = q;
        rho_t = kRhos[qt];
        // sector range: sum_{k > K} c_k rho_t^k <= (rho_t/rho)^K Z(rho) <= eps Z(rho_t)
        double best = INFINITY;
        for (int q = qt + 1; q < nv; ++q)
            best = fmin(best, (lz[q] - lz[qt] - log(kTailEps)) / log(kRhos[q] / rho_t));
        int K = isfinite(best) ? (int)ceil(best) : kMaxK;
        if (K < n) K = n;
        if (K > kMaxK) K = kMaxK;
        L = K + 1;
    }
    if (t == 0) {
        pl.pat_n[p] = n;
        pl.pat_L[p] = n < 0 ? 0 : L;
        pl.pat_rho[p] = rho_t;
        pl.unit_flag[p] = 0;
    }
    (void)order;
}

__global__ void approx_scan_kernel(int n_pat, long long cap, int n_single, ApproxPlan pl) {
    // one thread: patterns are few thousand at most per call
    if (threadIdx.x || blockIdx.x) return;
    long long run = 0;
    for (int p = 0; p < n_pat; ++p) {
        pl.unit_off[p] = run;
        int L = pl.pat_L[p];
        run += L > 0 ? (L / 2 + 1) : 0;
    }
    pl.unit_off[n_pat] = run;
    *pl.overflow = run > cap ? 1 : 0;
    *pl.total = run > cap ? 0 : run;
    int nmax = 0, Lmax = 1, nsmall = 0;
    long long secs = 0;
    for (int p = 0; p < n_pat; ++p) {
        nmax = pl.pat_n[p] > nmax ? pl.pat_n[p] : nmax;
        if (pl.pat_n[p] <= n_single && pl.pat_n[p] > nsmall) nsmall = pl.pat_n[p];
        Lmax = pl.pat_L[p] > Lmax ? pl.pat_L[p] : Lmax;
        pl.sec_off[p] = secs;
        secs += pl.pat_L[p] > 0 ? pl.pat_L[p] : 0;
    }
    pl.sec_off[n_pat] = secs;
    pl.info[0] = run;
    pl.info[1] = nmax;
    pl.info[2] = Lmax;
    pl.info[3] = secs;
    pl.info[4] = nsmall;  // largest n of the one-CTA minors kernel
}

// ---- minors at one nu point ------------------------------------------------------
// unpivoted LDL^T pivots of a complex symmetric K x K matrix (packed, in registers,
// K even); returns prod p^{-1/2}.  Every pivot of an accretive matrix has Re p > 0, so
// |arg p| < pi/2 and the principal root of a product of two pivots is the product of
// their principal roots: one root per pair of pivots.
template <typename R, int K>
__device__ __forceinline__ cx<R> ldl_rsqrt_prod(cx<R> (&a)[K * (K + 1) / 2], bool &bad) {
    cx<R> f = mk<R>(R(1), R(0)), prev = mk<R>(R(1), R(0));
#pragma unroll
    for (int k = 0; k < K; ++k) {
        cx<R> d = a[pidx(K, k, k)];
        if (!(d.re > R(0))) bad = true;
        if (k & 1) f = f * crsqrt(prev * d);
        prev = d;
        if (k + 1 < K) {
            cx<R> inv = cinv(d);
#pragma unroll
            for (int i = k + 1; i < K; ++i) {
                cx<R> li = a[pidx(K, k, i)] * inv;
#pragma unroll
                for (int j = i; j < K; ++j) a[pidx(K, i, j)] = cfms(a[pidx(K, i, j)], li, a[pidx(K, k, j)]);
            }
        }
    }
    return f;
}

// per-thread sums of the group terms: FP64 for FP64 minors; float-float (TwoSum) for
// FP32 minors, which keeps the FP64 pipe out of the inner loop
template <typename R> struct GroupAcc;
template <> struct GroupAcc<double> {
    double v[2 * (kMaxOrder + 1)];
    __device__ void zero() {
        for (int w = 0; w < 2 * (kMaxOrder + 1); ++w) v[w] = 0.0;
    }
    __device__ __forceinline__ void add(int w, cx<double> f) {
        v[2 * w] += f.re;
        v[2 * w + 1] += f.im;
    }
    __device__ __forceinline__ double get(int q) const { return v[q]; }
};
template <> struct GroupAcc<ff> {
    double v[2 * (kMaxOrder + 1)];
    __device__ void zero() {
        for (int w = 0; w < 2 * (kMaxOrder + 1); ++w) v[w] = 0.0;
    }
    __device__ __forceinline__ void add(int w, cx<ff> f) {
        v[2 * w] += ff_to_double(f.re);
        v[2 * w + 1] += ff_to_double(f.im);
    }
    __device__ __forceinline__ double get(int q) const { return v[q]; }
};
template <> struct GroupAcc<float> {
    float hi[2 * (kMaxOrder + 1)], lo[2 * (kMaxOrder + 1)];
    __device__ void zero() {
        for (int w = 0; w < 2 * (kMaxOrder + 1); ++w) hi[w] = lo[w] = 0.0f;
    }
    __device__ __forceinline__ void two(int q, float x) {
        const float s = hi[q] + x, bp = s - hi[q];
        lo[q] += (hi[q] - (s - bp)) + (x - bp);
        hi[q] = s;
    }
    __device__ __forceinline__ void add(int w, cx<float> f) {
        two(2 * w, f.re);
        two(2 * w + 1, f.im);
    }
    __device__ __forceinline__ double get(int q) const { return (double)hi[q] + (double)lo[q]; }
};

// G <- -(I - t O_S)^{-1} in shared memory (packed upper triangle of 2n x 2n, then four
// staged pivot columns of 2n entries), t = cs + i sn, by the symmetric sweep operator on
// every pivot; Z_S(t) = prod of principal pivot^{-1/2} (the LDL^T pivots, one root per
// pair) to s_zs on thread 0.  A pivot with Re <= 0 sets *s_bad.  All kMinorThreads threads
// take part; ends with a barrier.
template <typename R>
__device__ __forceinline__ void sweep_inverse(int M, const double *__restrict__ O, const int *modes, int n,
                                              double cs, double sn, cx<R> *G, int *s_bad, double *s_zs) {
    const int t = threadIdx.x;
    const int N = 2 * n, N2 = 2 * M;
    for (int f = t; f < N * N; f += kMinorThreads) {
        int i = f / N, j = f - i * N;
        if (j < i) continue;
        int si = modes[i >> 1] + (i & 1) * M, sj = modes[j >> 1] + (j & 1) * M;
        double o = O[(size_t)si * N2 + sj];
        G[pidx(N, i, j)] = init_entry<R>(i == j, cs, sn, o);
    }
    __syncthreads();
    // symmetric sweep operator on every pivot: G <- -(I - t O_S)^{-1};
    // Z_S(t) = prod of principal pivot^{-1/2} (pivots are the LDL^T pivots).
    // Pivot k's column is staged in cb (and cb / pivot in cu) by the previous pivot's
    // second phase, so an entry update is one complex product of staged values.
    cx<R> *const cb0 = G + sym(N), *const cb1 = cb0 + N, *const cu0 = cb0 + 2 * N, *const cu1 = cb0 + 3 * N;
    {
        const cx<R> inv0 = cinv(G[0]);
        for (int i = t; i < N; i += kMinorThreads) {
            const cx<R> v = G[pidx(N, 0, i)];
            cb0[i] = v;
            cu0[i] = v * inv0;
        }
    }
    __syncthreads();
    cx<double> zs = mk<double>(1.0, 0.0);
    cx<R> dprev = mk<R>(R(1), R(0));
    const int fw = N + 1, fE = (N >> 1) * fw;  // rows p and N - 1 - p folded: N + 1 entries
    for (int k = 0; k < N; ++k) {
        const cx<R> *cb = (k & 1) ? cb1 : cb0, *cu = (k & 1) ? cu1 : cu0;
        const cx<R> d = cb[k];
        if (!(d.re > R(0)) && t == 0) *s_bad = 1;
        if ((k & 1) && t == 0) zs = zs * widen(crsqrt(dprev * d));
        dprev = d;
        const cx<R> inv = cinv(d);
        int fp = t / fw, fq = t - fp * fw;
        const int sp = kMinorThreads / fw, sq = kMinorThreads - sp * fw;
        for (int f = t; f < fE; f += kMinorThreads) {
            int i, j;
            if (fq < N - fp) { i = fp; j = fp + fq; } else { i = N - 1 - fp; j = i + (fq - (N - fp)); }
            if (i != k && j != k) {
                cx<R> &e = G[i * N - (i * (i - 1)) / 2 + (j - i)];
                e = cfms_inl(e, cb[i], cu[j]);
            }
            fq += sq;
            fp += sp;
            if (fq >= fw) { fq -= fw; ++fp; }
        }
        __syncthreads();
        // scale pivot k's row and column; stage pivot k + 1's column
        cx<R> *cbn = (k & 1) ? cb0 : cb1, *cun = (k & 1) ? cu0 : cu1;
        const bool more = k + 1 < N;
        const cx<R> invn = more ? cinv(G[pidx(N, k + 1, k + 1)]) : mk<R>(R(0), R(0));
        for (int i = t; i < N; i += kMinorThreads) {
            if (i != k) G[pidx_any(N, i, k)] = cu[i];
            if (more) {
                // entry (k, k + 1) is the one just scaled: cu[k + 1]
                const cx<R> v = i == k ? cu[k + 1] : G[pidx_any(N, i, k + 1)];
                cbn[i] = v;
                cun[i] = v * invn;
            }
        }
        if (t == 0) G[pidx(N, k, k)] = mk<R>(R(0), R(0)) - inv;
        __syncthreads();
    }
    if (t == 0) { s_zs[0] = zs.re; s_zs[1] = zs.im; }
    __syncthreads();
}

// shared-memory entries of the one-CTA minors kernel for patterns of up to n clicks: the
// packed inverse, then max(the staged pivot columns, the pair phases' items); the items
// number at least n - 1 and up to 8 n as long as the CTAs per SM of the bare inverse stay
__host__ __device__ inline int minor_smem_entries(int n, int esz, int min_blocks) {
    constexpr long long kSM = 228 * 1024, kCTA = 227 * 1024, kPerCTA = 4 * 1024;  // 1 KB reserved + static
    const long long inv = (long long)n * (2 * n + 1), base = inv + 8LL * n;
    long long per = kSM / (min_blocks > 1 ? 2 : 1) - kPerCTA;
    if (base * esz > per) per = kCTA - kPerCTA;            // the inverse alone takes the SM
    long long items = (per / esz - inv) / 15;
    if (items > 8LL * n) items = 8LL * n;
    if (items < n - 1) items = n - 1;
    const long long ent = inv + (15 * items > 8LL * n ? 15 * items : 8LL * n);
    return (int)ent;
}

// Read-only view of the swept matrix -G, G = (I - t O_S)^{-1}, packed upper triangle of
// N x N: rows [0, rsplit) at b0, rows [rsplit, N) at b1 (whose first entry is packed
// entry off1).  One CTA: rsplit = N.  A CTA pair (cluster): each half in one CTA's shared
// memory, the other half reached through distributed shared memory.
template <typename R> struct GView {
    const cx<R> *b0, *b1;
    int N, rsplit, off1;
    __device__ __forceinline__ int rowoff(int r) const { return r * N - (r * (r - 1)) / 2 - r; }
    // p with p[col] = swept entry (r, col), col >= r
    __device__ __forceinline__ const cx<R> *row(int r) const {
        return r < rsplit ? b0 + rowoff(r) : b1 + (rowoff(r) - off1);
    }
    __device__ __forceinline__ cx<R> g(int i, int j) const {  // G(i, j) = -swept(i, j)
        const cx<R> v = i <= j ? row(i)[j] : row(j)[i];
        return mk<R>(-v.re, -v.im);
    }
};

// ---- the pair phases' items ------------------------------------------------------------
// Complex products, fused multiply-subtracts and roots: IN selects, for float-float, the
// inline forms of the shared out-of-line calls (the same operations).
template <typename R, bool IN> __device__ __forceinline__ cx<R> pmul(cx<R> a, cx<R> b) {
    if constexpr (IN) return cmul_ff(a, b); else return a * b;
}
template <typename R, bool IN> __device__ __forceinline__ cx<R> pfms(cx<R> e, cx<R> a, cx<R> b) {
    if constexpr (IN) return cfms_ff(e, a, b); else return cfms(e, a, b);
}
template <typename R, bool IN> __device__ __forceinline__ cx<R> prsqrt(cx<R> p) {
    if constexpr (IN) return crsqrt<ff>(p); else return crsqrt(p);
}
template <typename R, bool IN> __device__ __forceinline__ cx<R> pinv(cx<R> p) {
    if constexpr (IN) return cinv<ff>(p); else return cinv(p);
}
// item (b, e) of pair P = {a, b}: G_PP = L D L^T (unit lower L, accretive pivots), w = D^-1/2
// L^-1 G_{P,e}, H_e = G_ee - w^T w; stores w (8), H_e (3), H_e^-1 (3) and
// f3 = det(G_{P+e})^{-1/2} at o and returns f3 (bad: a pivot not accretive)
template <typename R> struct PairItem {
    cx<R> f3;
    int bad;
};
// G_PP = L D L^T of pair P = {a, b} (unit lower L, accretive pivots): L (6), D^-1/2 (4) and
// f2 = det(G_PP)^{-1/2} at pd[0..10]; returns 1 if a pivot is not accretive
constexpr int kPairLdl = 11;
template <typename R, bool IN>
__device__ __forceinline__ int pair_ldl_body(const GView<R> &V, int a, int b, cx<R> *pd) {
    int bad = 0;
    const int rr[4] = {2 * a, 2 * a + 1, 2 * b, 2 * b + 1};
    cx<R> m4[10];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = i; j < 4; ++j) m4[pidx(4, i, j)] = V.g(rr[i], rr[j]);
    cx<R> f2 = mk<R>(R(1), R(0)), prev = mk<R>(R(1), R(0));
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const cx<R> d = m4[pidx(4, k, k)];
        if (!(d.re > R(0))) bad = 1;
        if (k & 1) f2 = pmul<R, IN>(f2, prsqrt<R, IN>(pmul<R, IN>(prev, d)));
        prev = d;
        pd[6 + k] = prsqrt<R, IN>(d);
        const cx<R> inv = pinv<R, IN>(d);
#pragma unroll
        for (int i = k + 1; i < 4; ++i) {
            const cx<R> li = pmul<R, IN>(m4[pidx(4, k, i)], inv);
            pd[pidx(3, k, i - 1)] = li;
#pragma unroll
            for (int j = i; j < 4; ++j) m4[pidx(4, i, j)] = pfms<R, IN>(m4[pidx(4, i, j)], li, m4[pidx(4, k, j)]);
        }
    }
    pd[10] = f2;
    return bad;
}
// item (b, e) of pair P = {a, b} from the pair's factorisation pd: w = D^-1/2 L^-1 G_{P,e},
// H_e = G_ee - w^T w; stores w (8), H_e (3), H_e^-1 (3) and f3 = det(G_{P+e})^{-1/2} at o and
// returns f3 (bad: a pivot of H_e not accretive)
template <typename R, bool IN>
__device__ __forceinline__ PairItem<R> pair_item_from(const GView<R> &V, int a, int b, int e, const cx<R> *pd,
                                                      cx<R> *o) {
    PairItem<R> out;
    out.bad = 0;
    const int rr[4] = {2 * a, 2 * a + 1, 2 * b, 2 * b + 1};
    // y = L^-1 G_{P,e} (two columns), w = D^-1/2 y
    cx<R> w[4][2];
#pragma unroll
    for (int col = 0; col < 2; ++col) {
        cx<R> y[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            cx<R> v = V.g(rr[i], 2 * e + col);
#pragma unroll
            for (int k = 0; k < i; ++k) v = pfms<R, IN>(v, pd[pidx(3, k, i - 1)], y[k]);
            y[i] = v;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) w[i][col] = pmul<R, IN>(y[i], pd[6 + i]);
    }
    // H_e = G_ee - w^T w; its pivots h00 and det / h00
    cx<R> h00 = V.g(2 * e, 2 * e), h01 = V.g(2 * e, 2 * e + 1), h11 = V.g(2 * e + 1, 2 * e + 1);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        h00 = pfms<R, IN>(h00, w[k][0], w[k][0]);
        h01 = pfms<R, IN>(h01, w[k][0], w[k][1]);
        h11 = pfms<R, IN>(h11, w[k][1], w[k][1]);
    }
    const cx<R> det = pfms<R, IN>(pmul<R, IN>(h00, h11), h01, h01);
    if (!(h00.re > R(0)) || !(det.re * h00.re + det.im * h00.im > R(0))) out.bad = 1;
    out.f3 = pmul<R, IN>(pd[10], prsqrt<R, IN>(det));
    const cx<R> id = pinv<R, IN>(det);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        o[2 * k] = w[k][0];
        o[2 * k + 1] = w[k][1];
    }
    o[8] = h00;
    o[9] = h01;
    o[10] = h11;
    o[11] = pmul<R, IN>(h11, id);
    o[12] = mk<R>(R(0), R(0)) - pmul<R, IN>(h01, id);
    o[13] = pmul<R, IN>(h00, id);
    o[14] = out.f3;
    return out;
}
// item (b, e) with the pair's factorisation in registers (no table of them: the CTA pair)
template <typename R, bool IN>
__device__ __forceinline__ PairItem<R> pair_item_body(const GView<R> &V, int a, int b, int e, cx<R> *o) {
    cx<R> pd[kPairLdl];
    const int bad = pair_ldl_body<R, IN>(V, a, b, pd);
    PairItem<R> out = pair_item_from<R, IN>(V, a, b, e, pd, o);
    out.bad |= bad;
    return out;
}
template <typename R>
__device__ __forceinline__ PairItem<R> pair_item(const GView<R> &V, int a, int b, int e, cx<R> *o) {
    return pair_item_body<R, false>(V, a, b, e, o);
}
template <typename R> __device__ __forceinline__ int pair_ldl(const GView<R> &V, int a, int b, cx<R> *pd) {
    return pair_ldl_body<R, false>(V, a, b, pd);
}
template <typename R>
__device__ __forceinline__ PairItem<R> pair_item_tab(const GView<R> &V, int a, int b, int e, const cx<R> *pd,
                                                     cx<R> *o) {
    return pair_item_from<R, false>(V, a, b, e, pd, o);
}
// float-float: one out-of-line call per item (and per pair factorisation) with its
// arithmetic inline
static __device__ __noinline__ PairItem<ff> pair_item(const GView<ff> V, int a, int b, int e, cx<ff> *o) {
    return pair_item_body<ff, true>(V, a, b, e, o);
}
static __device__ __noinline__ int pair_ldl(const GView<ff> V, int a, int b, cx<ff> *pd) {
    return pair_ldl_body<ff, true>(V, a, b, pd);
}
static __device__ __noinline__ PairItem<ff> pair_item_tab(const GView<ff> V, int a, int b, int e, const cx<ff> *pd,
                                                          cx<ff> *o) {
    return pair_item_from<ff, true>(V, a, b, e, pd, o);
}

// The group terms det(G_WW)^{-1/2} of every W with |W| <= order, summed per |W| into acc.
// Groups of one and two detectors: worker `tid` of `nthr` takes every nthr-th.  Groups of
// three and four detectors go through each pair P = {a, b} (a < b) and the Schur
// complement of G_PP in G, G^(P) = G - G_.P G_PP^-1 G_P.: with H_e = G^(P)_ee (2 x 2),
//   det G_{P+e} = det G_PP det H_e,
//   det G_{P+c+d} = det G_PP det H_c det(H_d - K^T H_c^-1 K),  K = G^(P)_cd,
// and G^(P)_cd = G_cd - w_c^T w_d with w_e = D_P^-1/2 L_P^-1 G_Pe (G_PP = L_P D_P L_P^T).
// The pairs of one `a` are taken in groups of consecutive b: phase 1 stores w_e, H_e, H_e^-1
// and det(G_{P+e})^{-1/2} for every (b, e > b) of the group in `scratch` (cap items of 15
// complex entries; every CTA computes all of them with its own threads), phase 2 forms the
// four-detector terms of every (b, c, d), b < c < d (workers t2 of n2).  That is ~34 complex
// products per four-detector group, against ~60 through a 6 x 6 factorisation per triple.
// All pivots are accretive (Re > 0), so each determinant's principal root is the product of
// its factors' principal roots.  Every thread of the CTA must call this (it synchronises the
// CTA); s_off holds 2 (n + 1) ints of shared memory; add3: this CTA adds the three-detector
// terms (of a CTA pair, one computes them for its phase 2 only).  table: the group's pair
// factorisations G_PP = L D L^T are computed once per b into `scratch` ahead of the items
// (cap >= n - 1 then), instead of once per item.
template <typename R>
__device__ __forceinline__ void group_terms(const GView<R> &V, int n, int order, int tid, int nthr, int t2,
                                            int n2, cx<R> *scratch, int cap, int *s_off, bool add3, bool table,
                                            GroupAcc<R> &acc, bool &bad) {
    // w = 1: det of the 2x2 block, one root
    if (order >= 1)
        for (int a = tid; a < n; a += nthr) {
            cx<R> m[3] = {V.g(2 * a, 2 * a), V.g(2 * a, 2 * a + 1), V.g(2 * a + 1, 2 * a + 1)};
            acc.add(1, ldl_rsqrt_prod<R, 2>(m, bad));
        }
    // w = 2
    if (order >= 2)
        for (int idx = tid; idx < n * (n - 1) / 2; idx += nthr) {
            int a = 0, rem = idx;
            while (rem >= n - 1 - a) { rem -= n - 1 - a; ++a; }
            int b = a + 1 + rem;
            int rr[4] = {2 * a, 2 * a + 1, 2 * b, 2 * b + 1};
            cx<R> m[10];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = i; j < 4; ++j) m[pidx(4, i, j)] = V.g(rr[i], rr[j]);
            acc.add(2, ldl_rsqrt_prod<R, 4>(m, bad));
        }
    // order 4 in FP64 and float-float: the pair phases below; order 3, and every order in
    // FP32 (whose arithmetic is cheap next to the phases' barriers): a 6 x 6 factorisation
    // per triple, each serving its fourth detectors through a 2 x 2 Schur block
    constexpr bool kPairPhases = !std::is_same<R, float>::value;
    if (order >= 3 && !(kPairPhases && order >= 4)) {
        // w = 3, and w = 4 from each triple's factorisation.  Triples in order of their
        // largest detector c (then b, a), so the lanes of a warp share c and with it the
        // number n - 1 - c of fourth detectors d > c.
        if (order >= 3) {
            const long long ntri = (long long)n * (n - 1) * (n - 2) / 6;
            for (long long idx = tid; idx < ntri; idx += nthr) {
                // c: the largest with C(c, 3) <= idx; then b: the largest with C(b, 2) <= rem
                // (FP32 estimates on the MUFU pipe, corrected exactly in integers)
                int c = (int)cbrtf(6.0f * (float)idx);
                while ((long long)(c + 1) * c * (c - 1) / 6 <= idx) ++c;
                while ((long long)c * (c - 1) * (c - 2) / 6 > idx) --c;
                const long long rem = idx - (long long)c * (c - 1) * (c - 2) / 6;
                int b = (int)sqrtf(2.0f * (float)rem);
                while ((long long)(b + 1) * b / 2 <= rem) ++b;
                while ((long long)b * (b - 1) / 2 > rem) --b;
                const int a = (int)(rem - (long long)b * (b - 1) / 2);
                const int rr[6] = {2 * a, 2 * a + 1, 2 * b, 2 * b + 1, 2 * c, 2 * c + 1};
                // rows of the triple: entry (rr[i], col) with rr[i] <= col at rp[i][col]
                const cx<R> *rp[6];
    #pragma unroll
                for (int i = 0; i < 6; ++i) rp[i] = V.row(rr[i]);
                auto gr = [&](int i, int col) -> cx<R> { const cx<R> v = rp[i][col]; return mk<R>(-v.re, -v.im); };
                cx<R> w6[21];
    #pragma unroll
                for (int i = 0; i < 6; ++i)
    #pragma unroll
                    for (int j = i; j < 6; ++j) w6[pidx(6, i, j)] = gr(i, rr[j]);
                // LDL^T kept: unit lower L (Lf[k][i], k < i), inverse pivots Dinv
                cx<R> Lf[15], Dinv[6];
                cx<R> f3 = mk<R>(R(1), R(0)), prev = mk<R>(R(1), R(0));
    #pragma unroll
                for (int k = 0; k < 6; ++k) {
                    cx<R> d = w6[pidx(6, k, k)];
                    if (!(d.re > R(0))) bad = true;
                    if (k & 1) f3 = f3 * crsqrt(prev * d);
                    prev = d;
                    cx<R> inv = cinv(d);
                    Dinv[k] = inv;
    #pragma unroll
                    for (int i = k + 1; i < 6; ++i) {
                        cx<R> li = w6[pidx(6, k, i)] * inv;
                        Lf[pidx(5, k, i - 1)] = li;
    #pragma unroll
                        for (int j = i; j < 6; ++j) w6[pidx(6, i, j)] = cfms(w6[pidx(6, i, j)], li, w6[pidx(6, k, j)]);
                    }
                }
                acc.add(3, f3);
                // float-float: this triple's quads summed in float-float first, then one FP64
                // addition (keeps the FP64 pipe, 1/64 of FP32 here, out of the quad loop)
                constexpr bool kTriplePartial = std::is_same<R, ff>::value;
                cx<R> q4 = mk<R>(R(0), R(0));
                if (order >= 4)
                    for (int d4 = c + 1; d4 < n; ++d4) {
                        // y = L^{-1} G_{abc, d}; S = G_dd - y^T D^{-1} y (2 x 2); det S^{-1/2}
                        cx<R> y0[6], y1[6];
    #pragma unroll
                        for (int i = 0; i < 6; ++i) {
                            cx<R> v0 = gr(i, 2 * d4), v1 = gr(i, 2 * d4 + 1);
    #pragma unroll
                            for (int k = 0; k < i; ++k) {
                                v0 = cfms(v0, Lf[pidx(5, k, i - 1)], y0[k]);
                                v1 = cfms(v1, Lf[pidx(5, k, i - 1)], y1[k]);
                            }
                            y0[i] = v0;
                            y1[i] = v1;
                        }
                        const cx<R> *r0 = V.row(2 * d4), *r1 = V.row(2 * d4 + 1);
                        const cx<R> e00 = r0[2 * d4], e01 = r0[2 * d4 + 1], e11 = r1[2 * d4 + 1];
                        cx<R> s00 = mk<R>(-e00.re, -e00.im), s01 = mk<R>(-e01.re, -e01.im),
                              s11 = mk<R>(-e11.re, -e11.im);
    #pragma unroll
                        for (int k = 0; k < 6; ++k) {
                            const cx<R> z0 = y0[k] * Dinv[k], z1 = y1[k] * Dinv[k];
                            s00 = cfms(s00, z0, y0[k]);
                            s01 = cfms(s01, z0, y1[k]);
                            s11 = cfms(s11, z1, y1[k]);
                        }
                        // pivots s00 and det / s00 of the accretive block: Re > 0 each
                        const cx<R> det = cfms(s00 * s11, s01, s01);
                        if (!(s00.re > R(0)) || !(det.re * s00.re + det.im * s00.im > R(0))) bad = true;
                        const cx<R> term = f3 * crsqrt(det);
                        if constexpr (kTriplePartial) q4 = q4 + term;
                        else acc.add(4, term);
                    }
                if constexpr (kTriplePartial)
                    if (order >= 4) acc.add(4, q4);
            }
        }
    } else if (order >= 3 && n >= 3) {
        constexpr int IW = 15;  // per (b, e): w (4 x 2), H_e (3), H_e^-1 (3), det(G_{P+e})^{-1/2}
        const int t1 = threadIdx.x, n1 = blockDim.x;
        int *off1 = s_off, *off2 = s_off + (n + 1);
        cx<R> q4 = mk<R>(R(0), R(0));
        for (int a = 0; a + 2 < n; ++a) {
            for (int b0 = a + 1; b0 + 1 < n;) {
                // the group: b in [b0, b1) while its items (and with `table` each pair's
                // factorisation) fit in cap items' entries (at least one b: cap >= n - 2, and
                // n - 1 with the table)
                const int per_b = table ? kPairLdl : 0;
                int b1 = b0, items = 0;
                while (b1 + 1 < n &&
                       (b1 == b0 || IW * (items + (n - b1 - 1)) + per_b * (b1 - b0 + 1) <= IW * cap)) {
                    items += n - b1 - 1;
                    ++b1;
                }
                if (t1 == 0) {
                    int s1 = 0, s2 = 0;
                    for (int b = b0; b < b1; ++b) {
                        off1[b - b0] = s1;
                        off2[b - b0] = s2;
                        s1 += n - b - 1;
                        s2 += (n - b - 1) * (n - b - 2) / 2;
                    }
                    off1[b1 - b0] = s1;
                    off2[b1 - b0] = s2;
                }
                const int nb = b1 - b0;
                // the group's pair factorisations (with `table`), then its items
                cx<R> *const items_at = scratch + (size_t)per_b * nb;
                if (table)
                    for (int bb = t1; bb < nb; bb += n1)
                        if (pair_ldl(V, a, b0 + bb, scratch + (size_t)kPairLdl * bb)) bad = true;
                __syncthreads();
                // phase 1: every (b, e), e > b
                for (int it = t1; it < items; it += n1) {
                    int lo = 0, hi = nb;
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (off1[mid] <= it) lo = mid; else hi = mid;
                    }
                    const int b = b0 + lo, e = b + 1 + (it - off1[lo]);
                    const PairItem<R> pi = table ? pair_item_tab(V, a, b, e, scratch + (size_t)kPairLdl * lo,
                                                                 items_at + (size_t)IW * it)
                                                 : pair_item(V, a, b, e, items_at + (size_t)IW * it);
                    if (pi.bad) bad = true;
                    if (add3) acc.add(3, pi.f3);
                }
                __syncthreads();
                // phase 2: every (b, c, d), b < c < d
                if (order >= 4) {
                    const int total = off2[nb];
                    for (int it = t2; it < total; it += n2) {
                        int lo = 0, hi = nb;
                        while (hi - lo > 1) {
                            const int mid = (lo + hi) >> 1;
                            if (off2[mid] <= it) lo = mid; else hi = mid;
                        }
                        const int b = b0 + lo, r = it - off2[lo];
                        // (c', d') with c' < d' in colex order: r = d'(d' - 1)/2 + c'
                        int dp = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)r)) * 0.5f);
                        while (dp * (dp - 1) / 2 > r) --dp;
                        while ((dp + 1) * dp / 2 <= r) ++dp;
                        const int cp = r - dp * (dp - 1) / 2;
                        const int c = b + 1 + cp, d = b + 1 + dp;
                        const cx<R> *ic = items_at + (size_t)IW * (off1[lo] + cp);
                        const cx<R> *jd = items_at + (size_t)IW * (off1[lo] + dp);
                        // K = G^(P)_cd = G_cd - w_c^T w_d; X = H_c^-1 K; S = H_d - K^T X
                        const cx<R> k00 = rank4_entry(V.g(2 * c, 2 * d), ic, jd, 0, 0);
                        const cx<R> k01 = rank4_entry(V.g(2 * c, 2 * d + 1), ic, jd, 0, 1);
                        const cx<R> k10 = rank4_entry(V.g(2 * c + 1, 2 * d), ic, jd, 1, 0);
                        const cx<R> k11 = rank4_entry(V.g(2 * c + 1, 2 * d + 1), ic, jd, 1, 1);
                        const QuadTerm<R> qt = quad_term(k00, k01, k10, k11, ic, jd);
                        if (qt.bad) bad = true;
                        q4 = q4 + qt.term;
                    }
                }
                acc.add(4, q4);     // this group's four-detector terms (zero if order 3)
                q4 = mk<R>(R(0), R(0));
                __syncthreads();    // the group's items are read: the next group may overwrite them
                b0 = b1;
            }
        }
    }
}

// a warp's sums of the group terms (lanes combined by a fixed butterfly) into red[warp]
template <typename R>
__device__ __forceinline__ void warp_group_sums(const GroupAcc<R> &acc, double *red_row) {
    double accd[2 * (kMaxOrder + 1)];
#pragma unroll
    for (int w = 0; w < 2 * (kMaxOrder + 1); ++w) accd[w] = w < 2 ? 0.0 : acc.get(w);
#pragma unroll
    for (int w = 2; w < 2 * (kMaxOrder + 1); ++w)
        for (int off = 16; off; off >>= 1) accd[w] += __shfl_xor_sync(0xffffffffu, accd[w], off);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int w = 0; w < 2 * (kMaxOrder + 1); ++w) red_row[w] = accd[w];
}

// the unit's D_w(t_l) = Z_S(t_l) sum_{|W| = w} det(G_WW)^{-1/2}, from the warp sums in
// warp order (deterministic)
__device__ __forceinline__ void write_unit(const ApproxPlan &pl, long long u, int order, const double *zs,
                                           const double (*red)[2 * (kMaxOrder + 1)], int nwarps) {
    const cx<double> z = mk<double>(zs[0], zs[1]);
    double *out = pl.unit_D + (size_t)u * 2 * (kMaxOrder + 1);
    out[0] = z.re;
    out[1] = z.im;
    for (int w = 1; w <= kMaxOrder; ++w) {
        double re = 0.0, im = 0.0;
        for (int q = 0; q < nwarps; ++q) {
            re += red[q][2 * w];
            im += red[q][2 * w + 1];
        }
        cx<double> v = z * mk<double>(re, im);
        out[2 * w] = w <= order ? v.re : 0.0;
        out[2 * w + 1] = w <= order ? v.im : 0.0;
    }
}

// the pattern of unit u (skipping patterns without units: equal offsets)
__device__ __forceinline__ int unit_pattern(const ApproxPlan &pl, int n_pat, long long u) {
    int lo_ = 0, hi_ = n_pat;
    while (hi_ - lo_ > 1) {
        int mid = (lo_ + hi_) >> 1;
        if (pl.unit_off[mid] <= u) lo_ = mid; else hi_ = mid;
    }
    int p = lo_;
    while (p + 1 < n_pat && pl.unit_off[p + 1] <= u) ++p;
    return p;
}

// One CTA per (pattern, nu_l) unit, for patterns of up to n_single clicks (the packed
// inverse in this CTA's shared memory); larger patterns are left to the cluster kernel.
template <typename R>
__global__ void __launch_bounds__(kMinorThreads, MinorPrec<R>::min_blocks) approx_minors_kernel(int M, const double *__restrict__ O,
                                                                    const uint64_t *__restrict__ pats,
                                                                    int n_pat, int order, int n_single,
                                                                    int smem_entries,
                                                                    unsigned long long *counter,
                                                                    ApproxPlan pl) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<R> *G = (cx<R> *)smem_raw;
    __shared__ int modes[128];
    __shared__ int s_off[2 * (kApproxMaxN + 1)];
    __shared__ long long s_u;
    __shared__ int s_bad;
    __shared__ double red[kMinorThreads / 32][2 * (kMaxOrder + 1)];
    __shared__ double s_zs[2];
    const int t = threadIdx.x;
    const long long total = *pl.total;
    for (;;) {
        if (t == 0) s_u = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long u = s_u;
        if (u >= total) break;
        const int p = unit_pattern(pl, n_pat, u);
        const int l = (int)(u - pl.unit_off[p]);
        const int n = pl.pat_n[p], L = pl.pat_L[p];
        if (n > n_single) {   // a pattern for the CTA pairs
            __syncthreads();
            continue;
        }
        const uint64_t wlo = pats[2 * p], whi = pats[2 * p + 1];
        if (t == 0) {
            int c = 0;
            for (int i = 0; i < M; ++i) {
                uint64_t w = i < 64 ? wlo : whi;
                if (w >> (i & 63) & 1ull) modes[c++] = i;
            }
            s_bad = 0;
        }
        __syncthreads();
        const int N = 2 * n;
        // t = rho e^{i nu}, nu = 2 pi l / L; M_t = I - t O_S (complex symmetric)
        double sn, cs;
        sincospi(2.0 * (double)l / (double)L, &sn, &cs);
        const double rho = pl.pat_rho[p];
        sn *= rho;
        cs *= rho;
        sweep_inverse<R>(M, O, modes, n, cs, sn, G, &s_bad, s_zs);
        GroupAcc<R> acc;
        acc.zero();
        bool bad = false;
        const GView<R> V{G, G, N, N, 0};
        // the staged columns and the rest of the allocation serve the pair phases
        // items per group from this pattern's own n (not the batch's allocation): the work
        // split, and with it every rounding, is the same in any batch
        const int cap = (minor_smem_entries(n, (int)sizeof(cx<R>), MinorPrec<R>::min_blocks) - sym(N)) / 15;
        group_terms<R>(V, n, order, t, kMinorThreads, t, kMinorThreads, G + sym(N), cap, s_off, true, true, acc, bad);
        if (bad) s_bad = 1;
        warp_group_sums<R>(acc, red[t >> 5]);
        __syncthreads();
        if (t == 0) {
            write_unit(pl, u, order, s_zs, red, kMinorThreads / 32);
            if (s_bad) atomicOr(pl.unit_flag + p, 1);
        }
        __syncthreads();
    }
}

// ---- the same for large patterns on a CTA pair (thread-block cluster of two) ----------
// The packed 2n x 2n inverse of a pattern with n up to 112 clicks (403 KB in FP64 or
// float-float) exceeds one SM's shared memory: the two CTAs of a cluster hold half of its
// rows each and reach the other half through distributed shared memory.  The sweep
// operator runs on both halves at once (each CTA updates its own entries; the pivot
// columns are staged into both CTAs, one cluster barrier per pivot); the group terms are
// split over the 512 threads of the pair.
constexpr int kPairMaxN = kApproxMaxN;

// rows [0, rsplit) hold about half of the packed entries of an N x N upper triangle
__host__ __device__ inline int pair_split_row(int N) {
    const int half = (N * (N + 1) / 2 + 1) / 2;
    int r = 0, acc = 0;
    while (r < N && acc + (N - r) <= half) { acc += N - r; ++r; }
    return r > 0 ? r : 1;
}
__host__ __device__ inline int pair_part_entries(int N) {  // the larger half
    const int r = pair_split_row(N), lo = r * N - r * (r - 1) / 2, tot = N * (N + 1) / 2;
    return lo > tot - lo ? lo : tot - lo;
}

template <typename R>
__device__ void sweep_inverse_pair(cg::cluster_group &cl, int rank, int M, const double *__restrict__ O,
                                   const uint8_t *modes, int n, double cs, double sn, cx<R> *Gl, cx<R> *stage,
                                   cx<R> *stage_peer, int rsplit, int off1, int *s_bad, double *s_zs) {
    const int t = threadIdx.x;
    const int N = 2 * n, N2 = 2 * M;
    const int r_lo = rank ? rsplit : 0, r_hi = rank ? N : rsplit;
    const int base = rank ? off1 : 0;
    auto lidx = [&](int i, int j) { return i * N - (i * (i - 1)) / 2 + (j - i) - base; };  // own row i <= j
    for (int f = t; f < (r_hi - r_lo) * N; f += kMinorThreads) {
        const int i = r_lo + f / N, j = f - (f / N) * N;
        if (j < i) continue;
        const int si = modes[i >> 1] + (i & 1) * M, sj = modes[j >> 1] + (j & 1) * M;
        Gl[lidx(i, j)] = init_entry<R>(i == j, cs, sn, O[(size_t)si * N2 + sj]);
    }
    cx<R> *const cb0 = stage, *const cb1 = stage + N, *const cu = stage + 2 * N;
    cx<R> *const pb0 = stage_peer, *const pb1 = stage_peer + N;
    __syncthreads();
    // pivot 0's column is row 0: rank 0's
    if (rank == 0)
        for (int i = t; i < N; i += kMinorThreads) {
            const cx<R> v = Gl[lidx(0, i)];
            cb0[i] = v;
            pb0[i] = v;
        }
    cl.sync();
    cx<double> zs = mk<double>(1.0, 0.0);
    cx<R> dprev = mk<R>(R(1), R(0));
    // own rows folded in pairs (r_lo + q, r_hi - 1 - q): fw entries per pair
    const int nrows = r_hi - r_lo, npair = nrows >> 1, fw = 2 * N - r_lo - r_hi + 1, fE = npair * fw;
    const int sp = kMinorThreads / fw, sq = kMinorThreads - sp * fw;
    const int rmid = r_lo + npair;  // the unpaired middle row when nrows is odd
    for (int k = 0; k < N; ++k) {
        const cx<R> *cb = (k & 1) ? cb1 : cb0;
        cx<R> *cbn = (k & 1) ? cb0 : cb1, *pbn = (k & 1) ? pb0 : pb1;
        const cx<R> d = cb[k];
        if (!(d.re > R(0)) && t == 0) *s_bad = 1;
        if ((k & 1) && t == 0) zs = zs * widen(crsqrt(dprev * d));
        dprev = d;
        const cx<R> inv = cinv(d);
        for (int i = t; i < N; i += kMinorThreads) cu[i] = cb[i] * inv;
        __syncthreads();
        // entries (i, j), i, j != k, of the own rows: e -= cb_i cu_j
        int fp = t / fw, fq = t - fp * fw;
        for (int f = t; f < fE; f += kMinorThreads) {
            int i, j;
            const int a = r_lo + fp;
            if (fq < N - a) { i = a; j = a + fq; } else { i = r_hi - 1 - fp; j = i + (fq - (N - a)); }
            if (i != k && j != k) {
                cx<R> &e = Gl[lidx(i, j)];
                e = cfms_inl(e, cb[i], cu[j]);
            }
            fq += sq;
            fp += sp;
            if (fq >= fw) { fq -= fw; ++fp; }
        }
        if (nrows & 1)
            for (int j = rmid + t; j < N; j += kMinorThreads)
                if (rmid != k && j != k) {
                    cx<R> &e = Gl[lidx(rmid, j)];
                    e = cfms_inl(e, cb[rmid], cu[j]);
                }
        __syncthreads();
        // scale pivot k's row and column (own entries), stage pivot k + 1's column into
        // both CTAs (the owner of each entry writes it)
        const bool more = k + 1 < N;
        for (int i = t; i < N; i += kMinorThreads) {
            const int lo = i < k ? i : k, hi = i < k ? k : i;
            if (i != k && lo >= r_lo && lo < r_hi) Gl[lidx(lo, hi)] = cu[i];
            if (more) {
                const int l2 = i < k + 1 ? i : k + 1, h2 = i < k + 1 ? k + 1 : i;
                if (l2 >= r_lo && l2 < r_hi) {
                    // entry (k, k + 1) is the one just scaled: cu[k + 1]
                    const cx<R> v = i == k ? cu[k + 1] : Gl[lidx(l2, h2)];
                    cbn[i] = v;
                    pbn[i] = v;
                }
            }
        }
        if (t == 0 && k >= r_lo && k < r_hi) Gl[lidx(k, k)] = mk<R>(R(0), R(0)) - inv;
        cl.sync();
    }
    if (t == 0) { s_zs[0] = zs.re; s_zs[1] = zs.im; }
}

template <typename R>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kMinorThreads, 1)
approx_minors_pair_kernel(int M, const double *__restrict__ O, const uint64_t *__restrict__ pats, int n_pat,
                          int order, int n_single, int smem_entries, unsigned long long *counter, ApproxPlan pl) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint8_t modes[128];  // bytes: at 112 clicks the CTA needs all but ~0.2 KB of 227 KB
    __shared__ int s_off[2 * (kApproxMaxN + 1)];
    __shared__ long long s_u;
    __shared__ int s_bad;
    __shared__ double red[2 * (kMinorThreads / 32)][2 * (kMaxOrder + 1)];
    __shared__ double s_zs[2];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), t = threadIdx.x;
    const long long total = *pl.total;
    for (;;) {
        if (rank == 0 && t == 0) {
            const long long v = (long long)atomicAdd(counter, 1ull);
            s_u = v;
            *cl.map_shared_rank(&s_u, 1) = v;
        }
        cl.sync();
        const long long u = s_u;
        if (u >= total) break;
        const int p = unit_pattern(pl, n_pat, u);
        const int n = pl.pat_n[p];
        if (n <= n_single) {  // a pattern for the one-CTA kernel: both CTAs skip it
            cl.sync();        // (every thread has read s_u before rank 0 writes the next)
            continue;
        }
        const int l = (int)(u - pl.unit_off[p]), L = pl.pat_L[p];
        const uint64_t wlo = pats[2 * p], whi = pats[2 * p + 1];
        if (t == 0) {
            int c = 0;
            for (int i = 0; i < M; ++i) {
                uint64_t w = i < 64 ? wlo : whi;
                if (w >> (i & 63) & 1ull) modes[c++] = i;
            }
            s_bad = 0;
        }
        __syncthreads();
        const int N = 2 * n, rsplit = pair_split_row(N), off1 = rsplit * N - rsplit * (rsplit - 1) / 2;
        cx<R> *Gl = (cx<R> *)smem_raw;
        cx<R> *stage = Gl + pair_part_entries(N);
        cx<R> *stage_peer = cl.map_shared_rank(stage, rank ^ 1);
        double sn, cs;
        sincospi(2.0 * (double)l / (double)L, &sn, &cs);
        const double rho = pl.pat_rho[p];
        sn *= rho;
        cs *= rho;
        sweep_inverse_pair<R>(cl, rank, M, O, modes, n, cs, sn, Gl, stage, stage_peer, rsplit, off1, &s_bad, s_zs);
        cx<R> *G0 = rank == 0 ? Gl : cl.map_shared_rank(Gl, 0);
        cx<R> *G1 = rank == 1 ? Gl : cl.map_shared_rank(Gl, 1);
        const GView<R> V{G0, G1, N, rsplit, off1};
        GroupAcc<R> acc;
        acc.zero();
        bool bad = false;
        // each CTA computes every pair item in its own scratch (the staging area and beyond),
        // rank 0 adds the three-detector terms, the four-detector ones are split over both
        group_terms<R>(V, n, order, rank * kMinorThreads + t, 2 * kMinorThreads, rank * kMinorThreads + t,
                       2 * kMinorThreads, stage, n - 2, s_off, rank == 0, false, acc, bad);
        if (bad) s_bad = 1;
        // warp sums: rank 1's into rank 0's table (rows 8..15), then rank 0 writes the unit
        double (*red0)[2 * (kMaxOrder + 1)] = rank == 0 ? red : cl.map_shared_rank(red, 0);
        warp_group_sums<R>(acc, red0[rank * (kMinorThreads / 32) + (t >> 5)]);
        __syncthreads();
        if (rank == 1 && t == 0 && s_bad) atomicOr(cl.map_shared_rank(&s_bad, 0), 1);
        cl.sync();
        if (rank == 0 && t == 0) {
            write_unit(pl, u, order, s_zs, red, 2 * (kMinorThreads / 32));
            if (s_bad) atomicOr(pl.unit_flag + p, 1);
        }
        // the next ticket's barrier keeps both CTAs' shared memory live until the peer is done
    }
    cl.sync();
}

// ---- per-sector fit (maximum-entropy dual, damped Newton) ----------------------------
// One warp per sector: the lanes share the support points of the sums; every lane then
// takes the same Newton step from the same (broadcast) sums.
__device__ __forceinline__ double warp_sum_bcast(double v) {
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return __shfl_sync(0xffffffffu, v, 0);
}

// support x_s = v_s / n for v in [v0, n-1]; moments m (m_0 = 1); J + 1 coefficients
__device__ bool maxent_fit_warp(int v0, int n, int J, const double *m, double *a, int lane) {
    const int S = n - v0;
    auto phi_grad = [&](const double *aa, double *g, double *H, double &phi) {
        double pw[2 * kMaxOrder + 1];
        for (int q = 0; q <= 2 * J; ++q) pw[q] = 0.0;
        double ph = 0.0;
        for (int s = lane; s < S; s += 32) {
            double x = (double)(v0 + s) / n, f = 0.0, xp = 1.0;
            for (int i = 0; i <= J; ++i) { f += aa[i] * xp; xp *= x; }
            double q = exp(-f);
            ph += q;
            xp = 1.0;
            for (int i = 0; i <= 2 * J; ++i) { pw[i] += xp * q; xp *= x; }
        }
        phi = warp_sum_bcast(ph);
        for (int i = 0; i <= 2 * J; ++i) pw[i] = warp_sum_bcast(pw[i]);
        for (int i = 0; i <= J; ++i) {
            phi += aa[i] * m[i];
            if (g) g[i] = m[i] - pw[i];
            if (H)
                for (int k = 0; k <= J; ++k) H[i * (kMaxOrder + 1) + k] = pw[i + k];
        }
    };
    for (int i = 0; i <= J; ++i) a[i] = 0.0;
    a[0] = log((double)S);
    double g[kMaxOrder + 1], H[(kMaxOrder + 1) * (kMaxOrder + 1)], phi;
    phi_grad(a, g, H, phi);
    for (int it = 0; it < 200; ++it) {
        double gmax = 0.0;
        for (int i = 0; i <= J; ++i) gmax = fmax(gmax, fabs(g[i]));
        // H step = g by Gaussian elimination with partial pivoting (the Hessian is
        // positive definite but can be numerically singular for exact fits)
        double Ab[(kMaxOrder + 1) * (kMaxOrder + 2)], st[kMaxOrder + 1];
        const int W = kMaxOrder + 2;
        for (int i = 0; i <= J; ++i) {
            for (int k = 0; k <= J; ++k) Ab[i * W + k] = H[i * (kMaxOrder + 1) + k];
            Ab[i * W + J + 1] = g[i];
        }
        bool singular = false;
        for (int c = 0; c <= J && !singular; ++c) {
            int piv = c;
            for (int i = c + 1; i <= J; ++i)
                if (fabs(Ab[i * W + c]) > fabs(Ab[piv * W + c])) piv = i;
            if (Ab[piv * W + c] == 0.0) { singular = true; break; }
            if (piv != c)
                for (int k = 0; k <= J + 1; ++k) {
                    double tmp = Ab[c * W + k];
                    Ab[c * W + k] = Ab[piv * W + k];
                    Ab[piv * W + k] = tmp;
                }
            for (int i = c + 1; i <= J; ++i) {
                double f = Ab[i * W + c] / Ab[c * W + c];
                for (int k = c; k <= J + 1; ++k) Ab[i * W + k] -= f * Ab[c * W + k];
            }
        }
        if (singular) return gmax <= 1e-13;
        for (int i = J; i >= 0; --i) {
            double v = Ab[i * W + J + 1];
            for (int q = i + 1; q <= J; ++q) v -= Ab[i * W + q] * st[q];
            st[i] = v / Ab[i * W + i];
        }
        if (gmax <= 1e-13) {
            // a last full Newton step: the parameters converge, not only the moments
            for (int i = 0; i <= J; ++i) a[i] -= st[i];
            return true;
        }
        double gst = 0.0;
        for (int i = 0; i <= J; ++i) gst += g[i] * st[i];
        double tstep = 1.0, an[kMaxOrder + 1], gn[kMaxOrder + 1], Hn[(kMaxOrder + 1) * (kMaxOrder + 1)], phin;
        for (;;) {
            for (int i = 0; i <= J; ++i) an[i] = a[i] - tstep * st[i];
            phi_grad(an, gn, Hn, phin);
            if (isfinite(phin) && phin <= phi - 1e-4 * tstep * gst) break;
            double gnmax = 0.0;
            for (int i = 0; i <= J; ++i) gnmax = fmax(gnmax, fabs(gn[i]));
            if (isfinite(phin) && phin <= phi + 1e-14 * fabs(phi) && gnmax <= 0.5 * gmax) break;
            tstep *= 0.5;
            // no further decrease: moments on the boundary of the moment cone up to
            // their rounding; the fit stands if the residual is at that level
            if (tstep < 1e-12) return gmax <= 1e-10;
        }
        for (int i = 0; i <= J; ++i) { a[i] = an[i]; g[i] = gn[i]; }
        for (int i = 0; i < (kMaxOrder + 1) * (kMaxOrder + 1); ++i) H[i] = Hn[i];
        phi = phin;
    }
    double gmax = 0.0;
    for (int i = 0; i <= J; ++i) gmax = fmax(gmax, fabs(g[i]));
    return gmax <= 1e-10;
}

__device__ __forceinline__ double stirling2(int i, int w) {
    // S(i, w) for i, w <= 4
    const double tab[5][5] = {{1, 0, 0, 0, 0}, {0, 1, 0, 0, 0}, {0, 1, 1, 0, 0}, {0, 1, 3, 1, 0}, {0, 1, 7, 6, 1}};
    return tab[i][w];
}

// inverse DFT of one pattern's tables (real: O is real, so D(conj t) = conj D(t)):
//   D_w^(k) = (1/L) sum_l D_w(t_l) e^{-2 pi i k l / L},  one CTA per pattern
__global__ void __launch_bounds__(kDftThreads) approx_dft_kernel(int order, ApproxPlan pl) {
    extern __shared__ double tw[];  // cos, sin (2 pi m / L), m < L
    __shared__ double red[kDftThreads / 32];
    const int p = blockIdx.x, t = threadIdx.x;
    const int n = pl.pat_n[p], L = pl.pat_L[p];
    if (n < 0 || L <= 0 || *pl.overflow) return;
    const int H = L / 2;
    for (int m = t; m < L; m += kDftThreads) sincospi(2.0 * (double)m / (double)L, &tw[2 * m + 1], &tw[2 * m]);
    __syncthreads();
    const double *U = pl.unit_D + (size_t)pl.unit_off[p] * 2 * (kMaxOrder + 1);
    double *D = pl.sec_D + (size_t)pl.sec_off[p] * (kMaxOrder + 1);
    double mx = 0.0;
    for (int idx = t; idx < (order + 1) * L; idx += kDftThreads) {
        const int k = idx / (order + 1), w = idx - k * (order + 1);
        double s = U[2 * w];  // l = 0
        int m = 0;            // k l mod L
        for (int l = 1; l <= H; ++l) {
            m += k;
            if (m >= L) m -= L;
            const double re = U[(size_t)l * 2 * (kMaxOrder + 1) + 2 * w];
            const double im = U[(size_t)l * 2 * (kMaxOrder + 1) + 2 * w + 1];
            const double term = re * tw[2 * m] + im * tw[2 * m + 1];  // Re(D(t_l) e^{-i 2 pi k l / L})
            s += (2 * l == L) ? term : 2.0 * term;
        }
        D[(size_t)k * (kMaxOrder + 1) + w] = s / L;
        if (w == 0) mx = fmax(mx, s / L);
    }
    for (int off = 16; off; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((t & 31) == 0) red[t >> 5] = mx;
    __syncthreads();
    if (t == 0) {
        for (int w = 1; w < kDftThreads / 32; ++w) mx = fmax(mx, red[w]);
        pl.pat_max[p] = mx;
    }
}

// one warp per (pattern, sector k): factorial moments -> raw moments (Stirling numbers)
// -> maximum-entropy fit on the support v in [max(0, n - k), n - 1] -> the last point.
// curves (one pattern only, else null): every sector's fitted distribution over the
// clicks c = n - v, tilted, row k of curve_K + 1 rows of n + 1 (sectors with fewer photons
// than detectors are fitted too)
__global__ void __launch_bounds__(kSecThreads) approx_sector_fit_kernel(int n_pat, int order, double sector_eps,
                                                                      ApproxPlan pl, double *__restrict__ curves,
                                                                      int curve_K) {
    const int lane = threadIdx.x & 31;
    const long long nsec = pl.sec_off[n_pat];
    const long long nwarps = (long long)gridDim.x * (kSecThreads / 32);
    if (*pl.overflow) return;
    for (long long gs = (long long)blockIdx.x * (kSecThreads / 32) + (threadIdx.x >> 5); gs < nsec; gs += nwarps) {
        // the pattern whose sector range holds gs (the last with sec_off <= gs)
        int lo = 0, hi = n_pat;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (pl.sec_off[mid] <= gs) lo = mid; else hi = mid;
        }
        const int p = lo, n = pl.pat_n[p];
        const int k = (int)(gs - pl.sec_off[p]);
        const double *Dk = pl.sec_D + (size_t)gs * (kMaxOrder + 1);
        const double D0 = Dk[0];
        double val = 0.0;
        bool fell = false;
        const bool curve = curves != nullptr && k <= curve_K;
        if (curve && k == 0 && D0 > 0.0 && lane == 0) curves[0] = D0;   // no photon: no click (c = 0)
        if (n == 0) {
            val = (k == 0) ? D0 : 0.0;
        } else if ((k >= n || (curve && k >= 1)) && D0 >= sector_eps * pl.pat_max[p] && D0 > 0.0) {
            const int v0 = n - k > 0 ? n - k : 0;
            const int S = n - v0;
            const int Jmax = order < S - 1 ? order : S - 1;
            double mu[kMaxOrder + 1];
            for (int i = 0; i <= Jmax; ++i) {
                double s = 0.0, fw = 1.0;
                for (int w = 0; w <= i; ++w) {
                    s += stirling2(i, w) * fw * Dk[w];
                    fw *= (w + 1);
                }
                mu[i] = s;
            }
            bool done = false;
            for (int J = Jmax; J >= 0 && !done; --J) {
                double m[kMaxOrder + 1], a[kMaxOrder + 1];
                double np = 1.0;
                for (int i = 0; i <= J; ++i) { m[i] = mu[i] / np / mu[0]; np *= n; }
                if (maxent_fit_warp(v0, n, J, m, a, lane)) {
                    val = k >= n ? mu[0] * exp(-a[0]) : 0.0;
                    done = true;
                    if (J != Jmax) fell = true;
                    if (curve)
                        for (int v = v0 + lane; v < n; v += 32) {
                            const double x = (double)v / n;
                            double f = a[J];
                            for (int i = J - 1; i >= 0; --i) f = f * x + a[i];
                            curves[(size_t)k * (n + 1) + (n - v)] = mu[0] * exp(-f);
                        }
                }
            }
            if (!done) fell = true;
        }
        if (lane == 0) pl.sec_part[gs] = fell ? -val : val;   // the sign marks a fallback
    }
}

// the curves untilted (rho^-k) and scaled by det(sigma_Q)^{-1/2}
__global__ void approx_curve_scale_kernel(int curve_K, int n, const double *__restrict__ logdet, ApproxPlan pl,
                                          double *__restrict__ curves) {
    const long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= (long long)(curve_K + 1) * (n + 1)) return;
    const int k = (int)(f / (n + 1));
    curves[f] = *pl.overflow ? nan("") : curves[f] * exp(-0.5 * (*logdet) - k * log(pl.pat_rho[0]));
}

// per pattern (one warp): sum_k part_k rho^{-k} in logs (the tables are tilted by rho^k)
// floor_eps > 0 (FP32 minors, whose moments resolve sectors only down to that share of the
// largest): a sector k >= n below the floor carries at most floor_eps * (largest) of tilted
// mass, so its all-clicked point at most that; when those bounds add up to kFlagShare of the
// estimate, the estimate may be missing what the precision cannot resolve: GBS_E_FLOOR
__global__ void __launch_bounds__(kSumThreads) approx_sum_kernel(int n_pat, const double *__restrict__ logdet,
                                                               double floor_eps,
                                                               ApproxPlan pl, double *__restrict__ logP,
                                                               double *__restrict__ kappa,
                                                               double *__restrict__ err_bound,
                                                               int32_t *__restrict__ status) {
    const int p = blockIdx.x * (kSumThreads / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (p >= n_pat) return;
    const int n = pl.pat_n[p], L = pl.pat_L[p];
    if (n < 0 || *pl.overflow) {
        if (lane == 0) {
            logP[p] = nan("");
            if (kappa) kappa[p] = nan("");
            if (err_bound) err_bound[p] = nan("");
            if (status) status[p] = n < 0 ? GBS_E_INVALID : GBS_E_NOMEM;
        }
        return;
    }
    const double *part = pl.sec_part + pl.sec_off[p];
    const double lr = log(pl.pat_rho[p]);
    double top = -INFINITY;
    for (int k = lane; k < L; k += 32)
        if (part[k] != 0.0) top = fmax(top, log(fabs(part[k])) - k * lr);
    for (int off = 16; off; off >>= 1) top = fmax(top, __shfl_xor_sync(0xffffffffu, top, off));
    double s = 0.0, sf = 0.0, sd = 0.0;
    const double lfloor = floor_eps > 0.0 && pl.pat_max[p] > 0.0 ? log(floor_eps * pl.pat_max[p]) : -INFINITY;
    for (int k = lane; k < L; k += 32)
        if (part[k] != 0.0) {
            const double w = exp(log(fabs(part[k])) - k * lr - top);
            s += w;
            if (part[k] < 0.0) sf += w;
        } else if (k >= n && n > 0 && isfinite(lfloor)) {
            sd += exp(lfloor - k * lr - (isfinite(top) ? top : lfloor));
        }
    s = warp_sum_bcast(s);
    sf = warp_sum_bcast(sf);
    sd = warp_sum_bcast(sd);
    if (lane == 0) {
        logP[p] = s > 0.0 ? -0.5 * (*logdet) + top + log(s) : -INFINITY;
        if (kappa) kappa[p] = (double)(L - 1);
        if (err_bound) err_bound[p] = nan("");
        int st = GBS_OK;
        if (pl.unit_flag[p]) st = GBS_E_NOT_SPD;
        else if (sd > 0.0 && (!(s > 0.0) || sd >= kFlagShare * s)) st = GBS_E_FLOOR;
        else if (sf >= kFlagShare * s) st = GBS_E_FIT;
        if (status) status[p] = st;
    }
}

// ---- gradient of the approximation (not in the paper) ---------------------------------
// L = sum_p w_p log P_p; reverse mode through the steps above, per pattern:
//  * sum:     d log(sum_k part_k rho^-k) / d part_k = rho^-k / sum;
//  * fit:     implicit derivative of the moment conditions of the fitted exp(-f) on its
//             support, sum_s x_s^i F(x_s) = mu'_i with mu'_i = mu_i / n^i: at the solution
//             d part / d mu'_i = e^{-a_0} (Hn^-1)_0i, Hn_il = sum_s x_s^(i+l) e^{-f(x_s)} the
//             Newton matrix of the normalised fit;
//  * moments: mu'_i = sum_{w <= i} S(i, w) w! D_w^(k) / n^i;
//  * DFT:     D_w^(k) = (1/L) sum_{l <= L/2} c_l Re(D_w(t_l) e^{-2 pi i k l / L}), c_l = 1 for
//             l = 0 and l = L/2, else 2; the adjoint of D_w(t_l) as one complex number
//             (d/dRe - i d/dIm) is cbar_w(t_l) = (c_l / L) sum_k gamma_w^(k) e^{-2 pi i k l / L};
//  * minors:  with d det(X)^-1/2 = -1/2 det(X)^-1/2 tr(X^-1 dX) and I - t O = (1 - t) I + t A,
//             d Z_{S\W}(t) / dA_S = -1/2 t Z_{S\W}(t) [(I - t O_{S\W})^-1 embedded in S], and that
//             embedded inverse is G - G_{.W} G_WW^-1 G_{W.} (zero on the rows of W), so unit
//             (S, t_l) adds Re(-1/2 t (s G - G K G)) to dlog P / dA_S, with
//             s = sum_w cbar_w D_w(t) and K = sum_{W, |W| <= j} cbar_|W| Z_{S\W}(t) embed(G_WW^-1).
// K is built one 2 x 2 mode block (a, b) per warp (no atomics, a fixed summation order):
// every W holding a and b is V + {a, b} with V over the other modes; eliminating V first
// leaves on the rows of a and b the Schur complement of V in G_WW, whose inverse is the
// (a, b) block of G_WW^-1 and whose pivots complete det(G_WW).
constexpr int kGradApproxMaxN = 48;  // clicks per pattern on the approximation's gradient
constexpr int kPanel = 8;            // columns of K G per pass of the G K G product

__device__ __forceinline__ double factorial_small(int w) {
    const double tab[kMaxOrder + 1] = {1, 1, 2, 6, 24};
    return tab[w];
}

// y = Hn^-1 e_0 for the (J + 1) x (J + 1) Newton matrix Hn_il = pw[i + l] (Gaussian
// elimination with partial pivoting, as the fit's own step); false if singular
__device__ bool solve_e0(int J, const double *pw, double *y) {
    const int W = kMaxOrder + 2;
    double Ab[(kMaxOrder + 1) * (kMaxOrder + 2)];
    for (int i = 0; i <= J; ++i) {
        for (int k = 0; k <= J; ++k) Ab[i * W + k] = pw[i + k];
        Ab[i * W + J + 1] = i == 0 ? 1.0 : 0.0;
    }
    for (int c = 0; c <= J; ++c) {
        int piv = c;
        for (int i = c + 1; i <= J; ++i)
            if (fabs(Ab[i * W + c]) > fabs(Ab[piv * W + c])) piv = i;
        if (Ab[piv * W + c] == 0.0) return false;
        if (piv != c)
            for (int k = 0; k <= J + 1; ++k) {
                const double tmp = Ab[c * W + k];
                Ab[c * W + k] = Ab[piv * W + k];
                Ab[piv * W + k] = tmp;
            }
        for (int i = c + 1; i <= J; ++i) {
            const double f = Ab[i * W + c] / Ab[c * W + c];
            for (int k = c; k <= J + 1; ++k) Ab[i * W + k] -= f * Ab[c * W + k];
        }
    }
    for (int i = J; i >= 0; --i) {
        double v = Ab[i * W + J + 1];
        for (int q = i + 1; q <= J; ++q) v -= Ab[i * W + q] * y[q];
        y[i] = v / Ab[i * W + i];
    }
    return true;
}

// one warp per sector: the forward's fit again (same inputs and code, so the same order
// and coefficients), then beta_w = d part / d D_w^(k), w = 0..kMaxOrder (0 where unused)
__global__ void __launch_bounds__(kSecThreads) approx_fit_adjoint_kernel(int n_pat, int order, ApproxPlan pl,
                                                                       double *__restrict__ sec_B) {
    const int lane = threadIdx.x & 31;
    const long long nsec = pl.sec_off[n_pat];
    const long long nwarps = (long long)gridDim.x * (kSecThreads / 32);
    if (*pl.overflow) return;
    for (long long gs = (long long)blockIdx.x * (kSecThreads / 32) + (threadIdx.x >> 5); gs < nsec; gs += nwarps) {
        int lo = 0, hi = n_pat;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (pl.sec_off[mid] <= gs) lo = mid; else hi = mid;
        }
        const int p = lo, n = pl.pat_n[p];
        const int k = (int)(gs - pl.sec_off[p]);
        const double *Dk = pl.sec_D + (size_t)gs * (kMaxOrder + 1);
        double beta[kMaxOrder + 1];
        for (int w = 0; w <= kMaxOrder; ++w) beta[w] = 0.0;
        // fitted sectors only (k >= n: the support is v = 0..n-1)
        if (n > 0 && k >= n && pl.sec_part[gs] != 0.0) {
            const int Jmax = order < n - 1 ? order : n - 1;
            double mu[kMaxOrder + 1];
            for (int i = 0; i <= Jmax; ++i) {
                double s = 0.0, fw = 1.0;
                for (int w = 0; w <= i; ++w) {
                    s += stirling2(i, w) * fw * Dk[w];
                    fw *= (w + 1);
                }
                mu[i] = s;
            }
            for (int J = Jmax; J >= 0; --J) {
                double m[kMaxOrder + 1], a[kMaxOrder + 1];
                double np = 1.0;
                for (int i = 0; i <= J; ++i) { m[i] = mu[i] / np / mu[0]; np *= n; }
                if (!maxent_fit_warp(0, n, J, m, a, lane)) continue;
                double pw[2 * kMaxOrder + 1];
                for (int q = 0; q <= 2 * J; ++q) pw[q] = 0.0;
                for (int sp = lane; sp < n; sp += 32) {
                    const double x = (double)sp / n;
                    double f = 0.0, xp = 1.0;
                    for (int i = 0; i <= J; ++i) { f += a[i] * xp; xp *= x; }
                    const double q = exp(-f);
                    xp = 1.0;
                    for (int i = 0; i <= 2 * J; ++i) { pw[i] += xp * q; xp *= x; }
                }
                for (int i = 0; i <= 2 * J; ++i) pw[i] = warp_sum_bcast(pw[i]);
                double y[kMaxOrder + 1];
                if (solve_e0(J, pw, y)) {
                    const double e = exp(-a[0]);
                    for (int w = 0; w <= J; ++w) {
                        double s = 0.0, ni = 1.0;
                        for (int i = 0; i <= J; ++i) {
                            if (i >= w) s += y[i] * stirling2(i, w) * factorial_small(w) / ni;
                            ni *= n;
                        }
                        beta[w] = e * s;
                    }
                }
                break;
            }
        }
        if (lane == 0)
            for (int w = 0; w <= kMaxOrder; ++w) sec_B[(size_t)gs * (kMaxOrder + 1) + w] = beta[w];
    }
}

// one CTA per pattern: gamma_w^(k) = beta_w^(k) rho^-k / sum (in place), then the DFT's
// adjoint to the units: cbar_w(t_l), l = 0..L/2, interleaved (re, im) like unit_D
__global__ void __launch_bounds__(kDftThreads) approx_dft_adjoint_kernel(int order, ApproxPlan pl,
                                                                       double *__restrict__ sec_B,
                                                                       double *__restrict__ unit_B) {
    extern __shared__ double tw[];  // cos, sin (2 pi m / L), m < L
    __shared__ double s_top, s_sum;
    const int p = blockIdx.x, t = threadIdx.x;
    const int n = pl.pat_n[p], L = pl.pat_L[p];
    if (n <= 0 || L <= 0 || *pl.overflow) return;
    const int H = L / 2;
    const double *part = pl.sec_part + pl.sec_off[p];
    const double lr = log(pl.pat_rho[p]);
    if (t < 32) {
        // the sum of the tilted last points in logs, as the forward's sum
        double top = -INFINITY;
        for (int k = t; k < L; k += 32)
            if (part[k] != 0.0) top = fmax(top, log(fabs(part[k])) - k * lr);
        for (int off = 16; off; off >>= 1) top = fmax(top, __shfl_xor_sync(0xffffffffu, top, off));
        double s = 0.0;
        for (int k = t; k < L; k += 32)
            if (part[k] != 0.0) s += exp(log(fabs(part[k])) - k * lr - top);
        s = warp_sum_bcast(s);
        if (t == 0) { s_top = top; s_sum = s; }
    }
    for (int m = t; m < L; m += kDftThreads) sincospi(2.0 * (double)m / (double)L, &tw[2 * m + 1], &tw[2 * m]);
    __syncthreads();
    const double top = s_top, ssum = s_sum;
    double *B = sec_B + (size_t)pl.sec_off[p] * (kMaxOrder + 1);
    for (int k = t; k < L; k += kDftThreads) {
        const double gk = (part[k] != 0.0 && ssum > 0.0) ? exp(-k * lr - top) / ssum : 0.0;
        for (int w = 0; w <= kMaxOrder; ++w) B[(size_t)k * (kMaxOrder + 1) + w] *= gk;
    }
    __syncthreads();
    double *Ub = unit_B + (size_t)pl.unit_off[p] * 2 * (kMaxOrder + 1);
    for (int idx = t; idx < (H + 1) * (kMaxOrder + 1); idx += kDftThreads) {
        const int l = idx / (kMaxOrder + 1), w = idx - l * (kMaxOrder + 1);
        double re = 0.0, im = 0.0;
        if (w <= order) {
            int m = 0;  // k l mod L
            for (int k = 0; k < L; ++k) {
                const double gm = B[(size_t)k * (kMaxOrder + 1) + w];
                re += gm * tw[2 * m];
                im -= gm * tw[2 * m + 1];
                m += l;
                if (m >= L) m -= L;
            }
        }
        const double c = (l == 0 || 2 * l == L) ? 1.0 : 2.0;
        Ub[(size_t)l * 2 * (kMaxOrder + 1) + 2 * w] = c * re / L;
        Ub[(size_t)l * 2 * (kMaxOrder + 1) + 2 * w + 1] = c * im / L;
    }
}

// The modes m[0..NV-1] (V) and then the NT tail modes of G_WW (local mode indices, rows
// 2m and 2m + 1 of G), from the swept matrix Gs (= -G, packed): eliminate V's 2 NV pivots
// (unpivoted LDL^T) and return det(G_VV)^-1/2 (principal roots of pivot pairs; Re > 0
// for every pivot of the accretive G) with the Schur complement of V on the tail rows
// in s (packed 2 NT x 2 NT).
template <int NV, int NT>
__device__ __forceinline__ cx<double> schur_tail(const cx<double> *__restrict__ Gs, int N, const int (&m)[NV + NT],
                                                 cx<double> (&s)[NT * (2 * NT + 1)], bool &bad) {
    constexpr int K = 2 * (NV + NT);
    cx<double> a[K * (K + 1) / 2];
    int rr[K];
#pragma unroll
    for (int i = 0; i < K; ++i) rr[i] = 2 * m[i >> 1] + (i & 1);
#pragma unroll
    for (int i = 0; i < K; ++i)
#pragma unroll
        for (int j = i; j < K; ++j) {
            const cx<double> v = Gs[pidx_any(N, rr[i], rr[j])];
            a[pidx(K, i, j)] = mk<double>(-v.re, -v.im);
        }
    cx<double> f = mk<double>(1.0, 0.0), prev = mk<double>(1.0, 0.0);
#pragma unroll
    for (int k = 0; k < 2 * NV; ++k) {
        const cx<double> d = a[pidx(K, k, k)];
        if (!(d.re > 0.0)) bad = true;
        if (k & 1) f = f * crsqrt(prev * d);
        prev = d;
        const cx<double> inv = cinv(d);
#pragma unroll
        for (int i = k + 1; i < K; ++i) {
            const cx<double> li = a[pidx(K, k, i)] * inv;
#pragma unroll
            for (int j = i; j < K; ++j) a[pidx(K, i, j)] = a[pidx(K, i, j)] - li * a[pidx(K, k, j)];
        }
    }
#pragma unroll
    for (int i = 0; i < 2 * NT; ++i)
#pragma unroll
        for (int j = i; j < 2 * NT; ++j) s[pidx(2 * NT, i, j)] = a[pidx(K, 2 * NV + i, 2 * NV + j)];
    return f;
}

// C(o, v) for v <= 3
__device__ __forceinline__ int binom_small(int o, int v) {
    return v == 0 ? 1 : v == 1 ? o : v == 2 ? o * (o - 1) / 2 : o * (o - 1) * (o - 2) / 6;
}
// the r-th pair i1 < i2 in colex order (i2 the largest with C(i2, 2) <= r); FP32 estimate,
// corrected exactly in integers
__device__ __forceinline__ void unrank_pair(int r, int &i1, int &i2) {
    int c = (int)sqrtf(2.0f * (float)r);
    while ((c + 1) * c / 2 <= r) ++c;
    while (c * (c - 1) / 2 > r) --c;
    i2 = c;
    i1 = r - c * (c - 1) / 2;
}
// the r-th triple i1 < i2 < i3 in colex order
__device__ __forceinline__ void unrank_triple(int r, int &i1, int &i2, int &i3) {
    int c = (int)cbrtf(6.0f * (float)r);
    while ((c + 1) * c * (c - 1) / 6 <= r) ++c;
    while (c * (c - 1) * (c - 2) / 6 > r) --c;
    i3 = c;
    unrank_pair(r - c * (c - 1) * (c - 2) / 6, i1, i2);
}

// W = V + {a}: adds wz Z-factor det(G_WW)^-1/2 [G_WW^-1]_aa to the diagonal block (k00, k01, k11)
template <int NV>
__device__ __forceinline__ void diag_leaf(const cx<double> *__restrict__ Gs, int N, const int (&m)[NV + 1],
                                          cx<double> wz, cx<double> &k00, cx<double> &k01, cx<double> &k11,
                                          bool &bad) {
    cx<double> s[3];
    const cx<double> f = schur_tail<NV, 1>(Gs, N, m, s, bad);
    const cx<double> det = s[0] * s[2] - s[1] * s[1];
    if (!(s[0].re > 0.0) || !(det.re * s[0].re + det.im * s[0].im > 0.0)) bad = true;
    const cx<double> wgt = wz * f * crsqrt(det) * cinv(det);
    k00 = k00 + wgt * s[2];
    k01 = k01 - wgt * s[1];
    k11 = k11 + wgt * s[0];
}

// W = V + {a, b}, a < b: adds wz det(G_WW)^-1/2 [G_WW^-1]_ab to the off-diagonal block
// ko = (00, 01, 10, 11); with the tail S = [[P, Q], [Q^T, R]] (a's rows, b's rows),
// [S^-1]_ab = -P^-1 Q C^-1, C = R - Q^T P^-1 Q, det S = det P det C
template <int NV>
__device__ __forceinline__ void off_leaf(const cx<double> *__restrict__ Gs, int N, const int (&m)[NV + 2],
                                         cx<double> wz, cx<double> (&ko)[4], bool &bad) {
    cx<double> s[10];
    const cx<double> f = schur_tail<NV, 2>(Gs, N, m, s, bad);
    const cx<double> p00 = s[pidx(4, 0, 0)], p01 = s[pidx(4, 0, 1)], p11 = s[pidx(4, 1, 1)];
    const cx<double> q00 = s[pidx(4, 0, 2)], q01 = s[pidx(4, 0, 3)], q10 = s[pidx(4, 1, 2)], q11 = s[pidx(4, 1, 3)];
    const cx<double> r00 = s[pidx(4, 2, 2)], r01 = s[pidx(4, 2, 3)], r11 = s[pidx(4, 3, 3)];
    const cx<double> detP = p00 * p11 - p01 * p01;
    const cx<double> iP = cinv(detP);
    // X = P^-1 Q
    const cx<double> x00 = (p11 * q00 - p01 * q10) * iP, x01 = (p11 * q01 - p01 * q11) * iP;
    const cx<double> x10 = (p00 * q10 - p01 * q00) * iP, x11 = (p00 * q11 - p01 * q01) * iP;
    const cx<double> c00 = r00 - (q00 * x00 + q10 * x10), c01 = r01 - (q00 * x01 + q10 * x11),
                     c11 = r11 - (q01 * x01 + q11 * x11);
    const cx<double> detC = c00 * c11 - c01 * c01;
    const cx<double> iC = cinv(detC);
    if (!(p00.re > 0.0) || !(detP.re * p00.re + detP.im * p00.im > 0.0) || !(c00.re > 0.0) ||
        !(detC.re * c00.re + detC.im * c00.im > 0.0))
        bad = true;
    const cx<double> ci00 = c11 * iC, ci01 = mk<double>(0.0, 0.0) - c01 * iC, ci11 = c00 * iC;
    const cx<double> wgt = wz * f * crsqrt(detP) * crsqrt(detC);
    ko[0] = ko[0] - wgt * (x00 * ci00 + x01 * ci01);
    ko[1] = ko[1] - wgt * (x00 * ci01 + x01 * ci11);
    ko[2] = ko[2] - wgt * (x10 * ci00 + x11 * ci01);
    ko[3] = ko[3] - wgt * (x10 * ci01 + x11 * ci11);
}

// one CTA per (pattern, chunk of its contour points): per point t_l the inverse G (the
// forward's sweep), K block by block (a thread or a warp per block), then Re(-1/2 t (s G - G K G)) added to
// the chunk's own slot (packed upper triangle of 2n x 2n; every entry has one owner thread, so the
// sums over l are in a fixed order)
__global__ void __launch_bounds__(kMinorThreads, 1) approx_minors_adjoint_kernel(
    int M, const double *__restrict__ O, const uint64_t *__restrict__ pats, int order, int chunks_per,
    ApproxPlan pl, const double *__restrict__ unit_B, double *__restrict__ slots, size_t sst,
    int *__restrict__ flags) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int modes[128];
    __shared__ int s_bad;
    __shared__ double s_zs[2];
    const int t = threadIdx.x;
    const int p = blockIdx.x / chunks_per, c = blockIdx.x - p * chunks_per;
    const int n = pl.pat_n[p], L = pl.pat_L[p];
    if (n <= 0 || L <= 0 || *pl.overflow) return;
    const int N = 2 * n;
    cx<double> *const Gs = (cx<double> *)smem_raw;      // swept matrix, then four staged columns
    cx<double> *const Kp = Gs + sym(N) + 4 * N;          // K, packed upper triangle
    cx<double> *const Tp = Kp + sym(N);                  // N x kPanel columns of K G
    double *const slot = slots + (size_t)blockIdx.x * sst;
    for (int f = t; f < sym(N); f += kMinorThreads) slot[f] = 0.0;
    if (t == 0) {
        const uint64_t wlo = pats[2 * p], whi = pats[2 * p + 1];
        int q = 0;
        for (int i = 0; i < M; ++i) {
            const uint64_t w = i < 64 ? wlo : whi;
            if (w >> (i & 63) & 1ull) modes[q++] = i;
        }
        s_bad = 0;
    }
    __syncthreads();
    const int U = L / 2 + 1;
    const int l0 = (int)((long long)c * U / chunks_per), l1 = (int)((long long)(c + 1) * U / chunks_per);
    const double rho = pl.pat_rho[p];
    const int nb = n * (n + 1) / 2;
    bool bad = false;
    auto gt = [&](int i, int j) -> cx<double> { const cx<double> v = Gs[pidx_any(N, i, j)]; return mk<double>(-v.re, -v.im); };
    for (int l = l0; l < l1; ++l) {
        double sn, cs;
        sincospi(2.0 * (double)l / (double)L, &sn, &cs);
        sn *= rho;
        cs *= rho;
        sweep_inverse<double>(M, O, modes, n, cs, sn, Gs, &s_bad, s_zs);
        const size_t uo = ((size_t)pl.unit_off[p] + l) * 2 * (kMaxOrder + 1);
        cx<double> cb[kMaxOrder + 1];
        cx<double> sl = mk<double>(0.0, 0.0);
        for (int w = 0; w <= kMaxOrder; ++w) {
            cb[w] = mk<double>(unit_B[uo + 2 * w], unit_B[uo + 2 * w + 1]);
            sl = sl + cb[w] * mk<double>(pl.unit_D[uo + 2 * w], pl.unit_D[uo + 2 * w + 1]);
        }
        const cx<double> zs = mk<double>(s_zs[0], s_zs[1]);
        // one 2 x 2 block (a, b) per segment of gw lanes at a time: a thread at orders <= 2,
        // where a block holds few groups (an off-diagonal one a single group at order 2), a
        // warp above.  The segment's lanes split the block's groups W = V + {a, b}: V over the
        // other modes, sizes ascending and each size in colex order (neighbouring lanes mostly
        // share the size, so the leaf code rarely diverges); partial sums meet in a fixed
        // shuffle tree.  Every thread runs every round (the shuffles take the whole warp).
        const int gw = order <= 2 ? 1 : 32;
        const int seg = t / gw, sg = t - seg * gw, nseg = kMinorThreads / gw;
        const int rounds = (nb + nseg - 1) / nseg;
        for (int rd = 0; rd < rounds; ++rd) {
            const int blk = rd * nseg + seg;
            const bool live = blk < nb;
            int a = 0, rem = live ? blk : 0;
            while (rem >= n - a) { rem -= n - a; ++a; }
            const int b = a + rem;
            const bool dg = a == b;
            const int others = dg ? n - 1 : n - 2, base = dg ? 1 : 2;   // |W| = |V| + base
            const int vmax = order - base < others ? order - base : others;
            int cnt[4], total = 0;
            for (int v = 0; v < 4; ++v) {
                cnt[v] = live && v <= vmax ? binom_small(others, v) : 0;
                total += cnt[v];
            }
            const cx<double> z0 = mk<double>(0.0, 0.0);
            cx<double> acc[4] = {z0, z0, z0, z0};
            for (int q = sg; q < total; q += gw) {
                int v = 0, r = q;
                while (r >= cnt[v]) { r -= cnt[v]; ++v; }
                int x[3] = {r, 0, 0};
                if (v == 2) unrank_pair(r, x[0], x[1]);
                else if (v == 3) unrank_triple(r, x[0], x[1], x[2]);
                // ranks among the other modes -> modes (a, then b, skipped)
                for (int i = 0; i < v; ++i) {
                    int y = x[i];
                    if (y >= a) ++y;
                    if (!dg && y >= b) ++y;
                    x[i] = y;
                }
                const cx<double> wz = cb[v + base] * zs;
                if (dg) {
                    if (v == 0) {
                        const int m[1] = {a};
                        diag_leaf<0>(Gs, N, m, wz, acc[0], acc[1], acc[2], bad);
                    } else if (v == 1) {
                        const int m[2] = {x[0], a};
                        diag_leaf<1>(Gs, N, m, wz, acc[0], acc[1], acc[2], bad);
                    } else if (v == 2) {
                        const int m[3] = {x[0], x[1], a};
                        diag_leaf<2>(Gs, N, m, wz, acc[0], acc[1], acc[2], bad);
                    } else {
                        const int m[4] = {x[0], x[1], x[2], a};
                        diag_leaf<3>(Gs, N, m, wz, acc[0], acc[1], acc[2], bad);
                    }
                } else {
                    if (v == 0) {
                        const int m[2] = {a, b};
                        off_leaf<0>(Gs, N, m, wz, acc, bad);
                    } else if (v == 1) {
                        const int m[3] = {x[0], a, b};
                        off_leaf<1>(Gs, N, m, wz, acc, bad);
                    } else {
                        const int m[4] = {x[0], x[1], a, b};
                        off_leaf<2>(Gs, N, m, wz, acc, bad);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
                for (int off = gw >> 1; off; off >>= 1) {
                    acc[i].re += __shfl_xor_sync(0xffffffffu, acc[i].re, off);
                    acc[i].im += __shfl_xor_sync(0xffffffffu, acc[i].im, off);
                }
            if (live && sg == 0) {
                if (dg) {
                    Kp[pidx(N, 2 * a, 2 * a)] = acc[0];
                    Kp[pidx(N, 2 * a, 2 * a + 1)] = acc[1];
                    Kp[pidx(N, 2 * a + 1, 2 * a + 1)] = acc[2];
                } else {
                    Kp[pidx(N, 2 * a, 2 * b)] = acc[0];
                    Kp[pidx(N, 2 * a, 2 * b + 1)] = acc[1];
                    Kp[pidx(N, 2 * a + 1, 2 * b)] = acc[2];
                    Kp[pidx(N, 2 * a + 1, 2 * b + 1)] = acc[3];
                }
            }
        }
        __syncthreads();
        // Re(-1/2 t (s G - G K G)) on the upper triangle, kPanel columns at a time
        const cx<double> ht = mk<double>(-0.5 * cs, -0.5 * sn);
        for (int j0 = 0; j0 < N; j0 += kPanel) {
            for (int f = t; f < N * kPanel; f += kMinorThreads) {
                const int r = f / kPanel, j = j0 + (f - r * kPanel);
                cx<double> acc = mk<double>(0.0, 0.0);
                if (j < N)
                    for (int q = 0; q < N; ++q) acc = acc + Kp[pidx_any(N, r, q)] * gt(q, j);
                Tp[f] = acc;
            }
            __syncthreads();
            for (int f = t; f < N * kPanel; f += kMinorThreads) {
                const int i = f / kPanel, jj = f - i * kPanel, j = j0 + jj;
                if (j >= N || i > j) continue;
                cx<double> y = mk<double>(0.0, 0.0);
                for (int q = 0; q < N; ++q) y = y + gt(i, q) * Tp[q * kPanel + jj];
                const cx<double> v = ht * (sl * gt(i, j) - y);
                slot[pidx(N, i, j)] += v.re;
            }
            __syncthreads();
        }
    }
    if (bad) s_bad = 1;
    __syncthreads();
    if (t == 0 && s_bad) atomicOr(flags + p, 1);
}

// per pattern: F_p = w_p * (sum of its chunk slots, in chunk order), dense 2n x 2n at stride
// fst; zero for a pattern whose forward failed (status other than ok / fit fallback, or no
// sector) or whose adjoint met a non-positive pivot
__global__ void approx_grad_finalize_kernel(int chunks_per, ApproxPlan pl, const double *__restrict__ slots,
                                            size_t sst, const double *__restrict__ w,
                                            const double *__restrict__ logP, const int32_t *__restrict__ status,
                                            const int *__restrict__ flags, double *__restrict__ F, size_t fst) {
    const int p = blockIdx.x;
    const int n = pl.pat_n[p];
    if (n <= 0) return;
    const int D = 2 * n;
    const int st = status[p];
    const bool ok = (st == GBS_OK || st == GBS_E_FIT) && !flags[p] && isfinite(logP[p]);
    for (int f = threadIdx.x; f < D * D; f += blockDim.x) {
        const int i = f / D, j = f - i * D;
        double v = 0.0;
        if (ok) {
            const int q = pidx_any(D, i, j);
            for (int c = 0; c < chunks_per; ++c) v += slots[((size_t)p * chunks_per + c) * sst + q];
            v *= w[p];
        }
        F[(size_t)p * fst + f] = v;
    }
}

__global__ void approx_grad_status_kernel(int n_pat, const int32_t *__restrict__ st_in,
                                          const int *__restrict__ flags, int32_t *__restrict__ st_out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n_pat) st_out[p] = (st_in[p] == GBS_OK || st_in[p] == GBS_E_FIT) && flags[p] ? GBS_E_NOT_SPD : st_in[p];
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

struct ApproxOffsets {
    size_t counter, total, overflow, info, counter2, pat_n, pat_L, pat_rho, unit_off, unit_flag, sec_off, pat_max,
        unit_D, sec_D, sec_part, end;
};

ApproxOffsets approx_offsets(int n_pat, long long units, long long secs = 0) {
    ApproxOffsets o;
    o.counter = 0;
    o.total = 8;
    o.overflow = 16;
    o.info = 24;       // 6 long long
    o.counter2 = 72;   // the CTA-pair minors kernel's work counter
    o.pat_n = align256(80);
    o.pat_L = align256(o.pat_n + 4 * (size_t)n_pat);
    o.pat_rho = align256(o.pat_L + 4 * (size_t)n_pat);
    o.unit_off = align256(o.pat_rho + 8 * (size_t)n_pat);
    o.unit_flag = align256(o.unit_off + 8 * ((size_t)n_pat + 1));
    o.sec_off = align256(o.unit_flag + 4 * (size_t)n_pat);
    o.pat_max = align256(o.sec_off + 8 * ((size_t)n_pat + 1));
    o.unit_D = align256(o.pat_max + 8 * (size_t)n_pat);
    o.sec_D = align256(o.unit_D + 8 * 2 * (kMaxOrder + 1) * (size_t)units);
    o.sec_part = align256(o.sec_D + 8 * (kMaxOrder + 1) * (size_t)secs);
    o.end = o.sec_part + 8 * (size_t)secs;
    return o;
}

ApproxPlan approx_plan_from(void *ws, int n_pat, long long units = 0, long long secs = 0) {
    ApproxOffsets o = approx_offsets(n_pat, units, secs);
    char *b = (char *)ws;
    ApproxPlan pl;
    pl.total = (long long *)(b + o.total);
    pl.overflow = (int *)(b + o.overflow);
    pl.pat_n = (int *)(b + o.pat_n);
    pl.pat_L = (int *)(b + o.pat_L);
    pl.pat_rho = (double *)(b + o.pat_rho);
    pl.unit_off = (long long *)(b + o.unit_off);
    pl.unit_flag = (int *)(b + o.unit_flag);
    pl.unit_D = (double *)(b + o.unit_D);
    pl.info = (long long *)(b + o.info);
    pl.sec_off = (long long *)(b + o.sec_off);
    pl.pat_max = (double *)(b + o.pat_max);
    pl.sec_D = (double *)(b + o.sec_D);
    pl.sec_part = (double *)(b + o.sec_part);
    return pl;
}

template <typename R>
int run_approx(gbs_ctx *ctx, int M, const double *O, const double *logdet, const uint64_t *pats,
               int n_pat, int order, double *logP, double *kappa, double *err_bound, int32_t *status,
               double *curves = nullptr, int curve_K = -1, int curve_n = -1, int n_limit = -1) {
    // patterns up to this size are taken: the packed inverse must fit in one CTA's shared
    // memory, or (FP64 and float-float) in a CTA pair's; a caller may lower it
    const int n_cap = MinorPrec<R>::pair ? kPairMaxN : MinorPrec<R>::nmax;
    const int nmax_smem = n_limit > 0 && n_limit < n_cap ? n_limit : n_cap;
    const int n_single = MinorPrec<R>::pair && ctx->pair_from - 1 < MinorPrec<R>::nmax ? ctx->pair_from - 1
                                                                                       : MinorPrec<R>::nmax;
    static_assert(kMaxK + 1 <= 4096, "sector table");
    if (!ctx->ws || ctx->ws_bytes < approx_offsets(n_pat, 0).end) {
        int st = gbs_ws_ensure(ctx, approx_offsets(n_pat, 0).end);
        if (st) return st;
    }
    ApproxPlan pl = approx_plan_from(ctx->ws, n_pat);
    const size_t plan_smem = sizeof(double) * (size_t)sym(2 * kApproxMaxN);
    GBS_CUDA(ctx, cudaFuncSetAttribute(approx_plan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)plan_smem));
    const long long nocap = 1ll << 62;  // sized on the host below
    approx_plan_kernel<<<n_pat, kPlanThreads, plan_smem, ctx->stream>>>(M, O, pats, n_pat, order,
                                                                        nmax_smem, pl);
    GBS_CUDA(ctx, cudaGetLastError());
    approx_scan_kernel<<<1, 32, 0, ctx->stream>>>(n_pat, nocap, n_single, pl);
    GBS_CUDA(ctx, cudaGetLastError());
    // size the workspace and the kernels' shared memory from one readback (units,
    // largest n, largest L, sectors); re-plan if the workspace had to grow
    GBS_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, pl.info, 40, cudaMemcpyDeviceToHost, ctx->stream));
    GBS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const long long units = ((long long *)ctx->pinned)[0], secs = ((long long *)ctx->pinned)[3];
    const int nmax = (int)((long long *)ctx->pinned)[1], Lmax = (int)((long long *)ctx->pinned)[2];
    const int nsmall = (int)((long long *)ctx->pinned)[4];
    const size_t need = approx_offsets(n_pat, units, secs).end;
    if (need > ctx->ws_bytes) {
        int st = gbs_ws_ensure(ctx, need);
        if (st) return st;
        pl = approx_plan_from(ctx->ws, n_pat);
        approx_plan_kernel<<<n_pat, kPlanThreads, plan_smem, ctx->stream>>>(M, O, pats, n_pat, order,
                                                                            nmax_smem, pl);
        approx_scan_kernel<<<1, 32, 0, ctx->stream>>>(n_pat, nocap, n_single, pl);
        GBS_CUDA(ctx, cudaGetLastError());
    }
    pl = approx_plan_from(ctx->ws, n_pat, units, secs);
    GBS_CUDA(ctx, cudaMemsetAsync(ctx->ws, 0, 8, ctx->stream));  // work counters
    GBS_CUDA(ctx, cudaMemsetAsync((char *)ctx->ws + approx_offsets(n_pat, 0).counter2, 0, 8, ctx->stream));
    int st = gbs_timing_begin(ctx);
    if (st) return st;
    if (nsmall > 0) {
        // the packed inverse and four staged pivot columns, or the pair phases' items
        // (15 entries each, at least n - 1 of them, up to 8 n while the CTAs per SM stay)
        // (the largest over n <= nsmall: the kernel sizes each pattern's items from its own n,
        // and the floor to whole items makes the entries fall by up to 14 between some n)
        int ent = sym(2 * nsmall) + 8 * nsmall;  // FP32: no pair phases
        if constexpr (!std::is_same<R, float>::value)
            for (int m = 1; m <= nsmall; ++m) {
                const int e = minor_smem_entries(m, (int)sizeof(cx<R>), MinorPrec<R>::min_blocks);
                if (e > ent) ent = e;
            }
        const size_t minor_smem = sizeof(cx<R>) * (size_t)ent;
        GBS_CUDA(ctx, cudaFuncSetAttribute(approx_minors_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)minor_smem));
        int nb = 0;
        GBS_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, approx_minors_kernel<R>, kMinorThreads,
                                                                    minor_smem));
        if (nb < 1) nb = 1;
        approx_minors_kernel<R><<<ctx->num_sms * nb, kMinorThreads, minor_smem, ctx->stream>>>(
            M, O, pats, n_pat, order, n_single, ent, (unsigned long long *)ctx->ws, pl);
        GBS_CUDA(ctx, cudaGetLastError());
    }
    if constexpr (MinorPrec<R>::pair) if (nmax > n_single) {
        // half of the packed inverse, and three staged columns or the pair phases' items
        const int pent = pair_part_entries(2 * nmax) + (6 * nmax > 15 * (nmax - 2) ? 6 * nmax : 15 * (nmax - 2));
        const size_t pair_smem = sizeof(cx<R>) * (size_t)pent;
        GBS_CUDA(ctx, cudaFuncSetAttribute(approx_minors_pair_kernel<R>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pair_smem));
        approx_minors_pair_kernel<R><<<(ctx->num_sms / 2) * 2, kMinorThreads, pair_smem, ctx->stream>>>(
            M, O, pats, n_pat, order, n_single, pent,
            (unsigned long long *)((char *)ctx->ws + approx_offsets(n_pat, 0).counter2), pl);
        GBS_CUDA(ctx, cudaGetLastError());
    }
    st = gbs_timing_end(ctx);
    if (st) return st;
    const size_t dft_smem = sizeof(double) * 2 * (size_t)Lmax;
    GBS_CUDA(ctx, cudaFuncSetAttribute(approx_dft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)dft_smem));
    approx_dft_kernel<<<n_pat, kDftThreads, dft_smem, ctx->stream>>>(order, pl);
    GBS_CUDA(ctx, cudaGetLastError());
    const long long want = (secs + kSecThreads / 32 - 1) / (kSecThreads / 32);
    const int fit_blocks = (int)(want < (long long)ctx->num_sms * 16 ? (want > 0 ? want : 1) : ctx->num_sms * 16);
    if (curves) {
        // one pattern: its clicks (read back above) must be the caller's row width - 1
        if (nmax != curve_n)
            return gbs_fail(ctx, GBS_E_INVALID, "gbs_approx_sector_curves: the pattern has %d clicks, not n = %d",
                            nmax, curve_n);
        GBS_CUDA(ctx, cudaMemsetAsync(curves, 0, sizeof(double) * (size_t)(curve_K + 1) * (curve_n + 1),
                                      ctx->stream));
    }
    approx_sector_fit_kernel<<<fit_blocks, kSecThreads, 0, ctx->stream>>>(
        n_pat, order, MinorPrec<R>::sector_eps, pl, curves, curve_K);
    GBS_CUDA(ctx, cudaGetLastError());
    if (curves) {
        const long long tot = (long long)(curve_K + 1) * (nmax + 1);
        approx_curve_scale_kernel<<<(unsigned)((tot + 127) / 128), 128, 0, ctx->stream>>>(curve_K, nmax, logdet, pl,
                                                                                          curves);
        GBS_CUDA(ctx, cudaGetLastError());
    }
    approx_sum_kernel<<<(n_pat + kSumThreads / 32 - 1) / (kSumThreads / 32), kSumThreads, 0, ctx->stream>>>(
        n_pat, logdet, MinorPrec<R>::floor_flag ? MinorPrec<R>::sector_eps : 0.0, pl, logP, kappa, err_bound, status);
    GBS_CUDA(ctx, cudaGetLastError());
    return GBS_OK;
}

}  // namespace

int approx_prob(gbs_ctx *ctx, int M, const double *O, const double *logdet, const uint64_t *patterns,
                int n_pat, int order, int precision, double *logP, double *kappa, double *err_bound,
                int32_t *status) {
    if (order < 1 || order > kMaxOrder)
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_prob: approximation order %d not in 1..%d", order, kMaxOrder);
    if (precision == GBS_FP64)
        return run_approx<double>(ctx, M, O, logdet, patterns, n_pat, order, logP, kappa, err_bound, status);
    if (precision == GBS_FP32_SPLIT)
        return run_approx<float>(ctx, M, O, logdet, patterns, n_pat, order, logP, kappa, err_bound, status);
    if (precision == GBS_FF)
        return run_approx<ff>(ctx, M, O, logdet, patterns, n_pat, order, logP, kappa, err_bound, status);
    return gbs_fail(ctx, GBS_E_INVALID, "gbs_prob: the approximation runs in FP64, float-float or the FP32 split");
}

int approx_sector_curves(gbs_ctx *ctx, int M, const double *O, const double *logdet, const uint64_t *pattern,
                         int n, int order, int precision, int K, double *curves, double *logP, int32_t *status) {
    if (order < 1 || order > kMaxOrder)
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_approx_sector_curves: order %d not in 1..%d", order, kMaxOrder);
    if (n < 1 || n > M || K < 0)
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_approx_sector_curves: bad sizes (n=%d, M=%d, K=%d)", n, M, K);
    if (precision == GBS_FP64)
        return run_approx<double>(ctx, M, O, logdet, pattern, 1, order, logP, nullptr, nullptr, status, curves, K, n);
    if (precision == GBS_FF)
        return run_approx<ff>(ctx, M, O, logdet, pattern, 1, order, logP, nullptr, nullptr, status, curves, K, n);
    return gbs_fail(ctx, GBS_E_INVALID, "gbs_approx_sector_curves: the curves run in FP64 or float-float");
}

int approx_grad(gbs_ctx *ctx, int M, const double *O, const double *logdet, const uint64_t *pats, int n_pat,
                int order, const double *w, double *dsq, double *logP, int32_t *status) {
    if (order < 1 || order > kMaxOrder)
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_grad_approx: order %d not in 1..%d", order, kMaxOrder);
    // every pattern must be valid with at most kGradApproxMaxN clicks: checked on the host
    // from a copy of the pattern words (one small readback)
    const size_t pb = (size_t)n_pat * 16;
    uint64_t *hp = (uint64_t *)malloc(pb + 16);
    if (!hp) return gbs_fail(ctx, GBS_E_NOMEM, "gbs_grad_approx: host buffer");
    cudaError_t ce = cudaMemcpyAsync(hp, pats, pb, cudaMemcpyDeviceToHost, ctx->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
    if (ce != cudaSuccess) {
        free(hp);
        GBS_CUDA(ctx, ce);
    }
    int n_max = 0;
    for (int p = 0; p < n_pat; ++p) {
        const uint64_t lo = hp[2 * p], hi = hp[2 * p + 1];
        const int n = __builtin_popcountll(lo) + __builtin_popcountll(hi);
        const bool out_of_range =
            (M < 64 && (lo >> M)) || (M <= 64 && hi) || (M > 64 && M < 128 && (hi >> (M - 64)));
        if (n > kGradApproxMaxN || out_of_range) {
            free(hp);
            return gbs_fail(ctx, GBS_E_INVALID,
                            "gbs_grad_approx: pattern %d has %d clicks (at most %d) or a detector >= M", p, n,
                            kGradApproxMaxN);
        }
        n_max = n > n_max ? n : n_max;
    }
    free(hp);
    // kept across the forward: its log P and status, the adjoint's flags
    const size_t np_ = (size_t)n_pat;
    const size_t o_lp = 0, o_st = align256(8 * np_), o_fl = o_st + align256(4 * np_), keep = o_fl + align256(4 * np_);
    int st = gbs_aux_ensure(ctx, keep, 0);
    if (st) return st;
    {
        char *b = (char *)ctx->aux;
        st = run_approx<double>(ctx, M, O, logdet, pats, n_pat, order, (double *)(b + o_lp), nullptr, nullptr,
                                (int32_t *)(b + o_st), nullptr, -1, -1, kGradApproxMaxN);
        if (st) return st;
    }
    // the plan's sizes (units, largest n, largest L, sectors)
    ApproxPlan pl = approx_plan_from(ctx->ws, n_pat);
    GBS_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, pl.info, 32, cudaMemcpyDeviceToHost, ctx->stream));
    GBS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const long long units = ((long long *)ctx->pinned)[0], secs = ((long long *)ctx->pinned)[3];
    const int Lmax = (int)((long long *)ctx->pinned)[2];
    pl = approx_plan_from(ctx->ws, n_pat, units, secs);
    // contour points of a pattern split over chunks_per CTAs: about two CTAs per SM in all
    const int want = (2 * ctx->num_sms + n_pat - 1) / n_pat;
    const int chunks_per = want < 1 ? 1 : (want > 64 ? 64 : want);
    const int Nm = 2 * (n_max > 0 ? n_max : 1);
    const size_t sst = (size_t)sym(Nm), fst = (size_t)Nm * Nm, N2 = (size_t)(2 * M) * (2 * M);
    const size_t o_sb = keep, o_ub = o_sb + align256(8 * (kMaxOrder + 1) * (size_t)secs),
                 o_sl = o_ub + align256(16 * (kMaxOrder + 1) * (size_t)units),
                 o_F = o_sl + align256(8 * np_ * chunks_per * sst), o_H = o_F + align256(8 * np_ * fst),
                 o_T1 = o_H + align256(8 * N2), o_T2 = o_T1 + align256(8 * N2), o_sw = o_T2 + align256(8 * N2),
                 total = o_sw + 256;
    st = gbs_aux_ensure(ctx, total, keep);
    if (st) return st;
    char *b = (char *)ctx->aux;
    double *lp_i = (double *)(b + o_lp);
    int32_t *st_i = (int32_t *)(b + o_st);
    int *flags = (int *)(b + o_fl);
    double *sec_B = (double *)(b + o_sb), *unit_B = (double *)(b + o_ub), *slots = (double *)(b + o_sl);
    double *F = (double *)(b + o_F), *H = (double *)(b + o_H), *T1 = (double *)(b + o_T1), *T2 = (double *)(b + o_T2),
           *sw = (double *)(b + o_sw);
    GBS_CUDA(ctx, cudaMemsetAsync(flags, 0, 4 * np_, ctx->stream));
    if (secs > 0) {
        const long long wsec = (secs + kSecThreads / 32 - 1) / (kSecThreads / 32);
        const int fit_blocks = (int)(wsec < (long long)ctx->num_sms * 16 ? wsec : ctx->num_sms * 16);
        approx_fit_adjoint_kernel<<<fit_blocks, kSecThreads, 0, ctx->stream>>>(n_pat, order, pl, sec_B);
        GBS_CUDA(ctx, cudaGetLastError());
        const size_t dft_smem = sizeof(double) * 2 * (size_t)(Lmax > 0 ? Lmax : 1);
        GBS_CUDA(ctx, cudaFuncSetAttribute(approx_dft_adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)dft_smem));
        approx_dft_adjoint_kernel<<<n_pat, kDftThreads, dft_smem, ctx->stream>>>(order, pl, sec_B, unit_B);
        GBS_CUDA(ctx, cudaGetLastError());
    }
    if (n_max > 0) {
        // swept matrix + four staged columns, K, one panel of K G
        const size_t smem = sizeof(cx<double>) * (2 * sst + 4 * (size_t)Nm + (size_t)Nm * kPanel);
        GBS_CUDA(ctx, cudaFuncSetAttribute(approx_minors_adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem));
        approx_minors_adjoint_kernel<<<(unsigned)(n_pat * chunks_per), kMinorThreads, smem, ctx->stream>>>(
            M, O, pats, order, chunks_per, pl, unit_B, slots, sst, flags);
        GBS_CUDA(ctx, cudaGetLastError());
        approx_grad_finalize_kernel<<<n_pat, 256, 0, ctx->stream>>>(chunks_per, pl, slots, sst, w, lp_i, st_i, flags,
                                                                   F, fst);
        GBS_CUDA(ctx, cudaGetLastError());
    }
    st = grad_chain_sigma(ctx, M, O, pats, n_pat, F, fst, w, H, T1, T2, sw, dsq);
    if (st) return st;
    if (logP) GBS_CUDA(ctx, cudaMemcpyAsync(logP, lp_i, 8 * np_, cudaMemcpyDeviceToDevice, ctx->stream));
    if (status) {
        // a pattern the adjoint could not differentiate reports GBS_E_NOT_SPD
        approx_grad_status_kernel<<<(n_pat + 255) / 256, 256, 0, ctx->stream>>>(n_pat, st_i, flags, status);
        GBS_CUDA(ctx, cudaGetLastError());
    }
    return GBS_OK;
}
