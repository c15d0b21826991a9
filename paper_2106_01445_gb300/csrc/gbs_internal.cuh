// Internal declarations shared by the translation units of libgbs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/gbs.h"

struct gbs_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    char err[512] = {0};
    // device workspace (grown on demand, or pre-sized by gbs_reserve)
    void *ws = nullptr;
    size_t ws_bytes = 0;
    bool reserved = false;
    long long cap_units = 0;  // unit partial slots in the workspace
    int cap_pat = 0;          // patterns covered by the workspace
    // pinned host scratch for small readbacks, and a small device scratch
    void *pinned = nullptr;
    int32_t *dscratch = nullptr;
    // buffers of gbs_run_host (device copies of the host inputs)
    void *host_io = nullptr;
    size_t host_io_bytes = 0;
    // GBS_AUTO: the double-double rerun's patterns and outputs
    void *aux = nullptr;
    size_t aux_bytes = 0;
    // persistent-grid sizes of the sweep kernels (CTAs per SM), by precision
    int sweep_blocks_per_sm[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    // prefix levels looped inside one sweep unit, by precision (-1: the default);
    // set by gbs_autotune
    int sweep_split[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
    // approximation: patterns of at least this many clicks take the CTA-pair minors kernel
    // (FP64 and float-float; above 79 clicks they must)
    int pair_from = 80;
    // optional event timing of the sweep kernel launches
    static const int kTimingRing = 4096;
    bool timing = false;
    cudaEvent_t *tev = nullptr;   // 2 * kTimingRing events
    long long t_head = 0, t_tail = 0;
    double t_ms = 0.0;
    long long t_launches = 0;
};

// Bracket one sweep launch with timing events (no-ops unless timing is on).
int gbs_timing_begin(gbs_ctx *ctx);
int gbs_timing_end(gbs_ctx *ctx);

// Record an error message on the context and return the code.
int gbs_fail(gbs_ctx *ctx, int code, const char *fmt, ...);

#define GBS_CUDA(ctx, call)                                                                  \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return gbs_fail((ctx), GBS_E_CUDA, "%s failed: %s (%s:%d)", #call,              \
                            cudaGetErrorString(e_), __FILE__, __LINE__);                      \
    } while (0)

// Grow the context workspace to at least `bytes` (synchronises the stream).
int gbs_ws_ensure(gbs_ctx *ctx, size_t bytes);
// Grow the auxiliary buffer to at least `bytes`, keeping its first `keep` bytes
// (synchronises the stream when it grows).
int gbs_aux_ensure(gbs_ctx *ctx, size_t bytes, size_t keep);

// --- launchers implemented in the kernel translation units ---------------
int launch_build_state(gbs_ctx *ctx, int M, const double *U, const double *r, double eta,
                       double *sigma, double *O, double *logdet, int32_t *status_dev);
int launch_gen_patterns(gbs_ctx *ctx, uint64_t seed, uint32_t stream, int M, int n_lo,
                        int n_hi, int n_pat, uint64_t *out);
int sweep_exact(gbs_ctx *ctx, int M, const double *O, const double *logdet,
                const uint64_t *patterns, int n_pat, int precision, double *logP,
                double *kappa, double *err_bound, int32_t *status);
int sweep_exact_on(gbs_ctx *ctx, void *ws, size_t ws_bytes, int M, const double *O,
                   const double *logdet, const uint64_t *patterns, int n_pat, int precision,
                   double *logP, double *kappa, double *err_bound, int32_t *status);
size_t sweep_workspace_bytes(int n_pat, long long units);
size_t sweep_workspace_bytes_prec(int n_pat, long long units, int precision);
int sweep_slice(gbs_ctx *ctx, int M, const double *O, const uint64_t *patterns, int n_pat, int precision,
                int part, int nparts, double *partial, int32_t *pflag);
int sweep_combine(gbs_ctx *ctx, const double *logdet, const uint64_t *patterns, int n_pat, int precision,
                  int nparts, const double *partials, const int32_t *pflags, double *logP, double *kappa,
                  double *err_bound, int32_t *status);
long long sweep_units_upper_bound(int n_pat, int n_max, int precision, int split);
int sweep_split_of(const gbs_ctx *ctx, int precision);
int sweep_auto(gbs_ctx *ctx, int M, const double *O, const double *logdet, const uint64_t *patterns, int n_pat,
               double *logP, double *kappa, double *err_bound, int32_t *status);
size_t sweep_auto_bytes(int n_pat);
int click_distribution(gbs_ctx *ctx, int M, const double *O, const double *logdet, double *logp,
                       double *kappa);
int sector_distribution(gbs_ctx *ctx, int M, const double *O, const double *logdet, int L, double rho, int K,
                        int even, int precision, double *pkn);
int approx_prob(gbs_ctx *ctx, int M, const double *O, const double *logdet, const uint64_t *patterns,
                int n_pat, int order, int precision, double *logP, double *kappa, double *err_bound,
                int32_t *status);
int approx_sector_curves(gbs_ctx *ctx, int M, const double *O, const double *logdet, const uint64_t *pattern,
                         int n, int order, int precision, int K, double *curves, double *logP, int32_t *status);
int approx_grad(gbs_ctx *ctx, int M, const double *O, const double *logdet, const uint64_t *pats, int n_pat,
                int order, const double *w, double *dsq, double *logP, int32_t *status);
// dL/dsigma_Q = -1/2 (sum w) A - A H A, H the per-pattern F_p (dense 2n x 2n at stride fst,
// rows in the order of the clicked modes, x and p interleaved) embedded in 2M x 2M;
// scratch H, T1, T2 (2M x 2M) and sw (one double)
int grad_chain_sigma(gbs_ctx *ctx, int M, const double *O, const uint64_t *pats, int n_pat, const double *F,
                     size_t fst, const double *w, double *H, double *T1, double *T2, double *sw, double *dsq);
int grad_sigmaQ(gbs_ctx *ctx, int M, const double *O, const double *logdet, const uint64_t *pats,
                int n_pat, const double *w, double *dsq, double *logP, int32_t *status);
int grad_params(gbs_ctx *ctx, int M, const double *U, const double *r, double eta, const double *dsq,
                double *dU, double *dr, double *deta);
int clements_unitary(gbs_ctx *ctx, int M, const double *theta, const double *phi, double *U);
int clements_grad(gbs_ctx *ctx, int M, const double *theta, const double *phi, const double *U,
                  const double *dU, double *dtheta, double *dphi);
int peak_flops(gbs_ctx *ctx, int kind, double *flops);
