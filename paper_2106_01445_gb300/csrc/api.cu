// C ABI entry points of libgbs: context, workspace and argument checks.
// The arithmetic lives in state.cu, gen.cu and sweep.cu.
#include <stdarg.h>
#include <stdlib.h>
#include <string.h>

#include "gbs_internal.cuh"

int gbs_fail(gbs_ctx *ctx, int code, const char *fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

int gbs_ws_ensure(gbs_ctx *ctx, size_t bytes) {
    if (bytes <= ctx->ws_bytes) return GBS_OK;
    GBS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->ws) GBS_CUDA(ctx, cudaFree(ctx->ws));
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
    size_t want = bytes + bytes / 4 + (1 << 20);
    if (cudaMalloc(&ctx->ws, want) != cudaSuccess) {
        cudaGetLastError();
        return gbs_fail(ctx, GBS_E_NOMEM, "cannot allocate %zu bytes of workspace", want);
    }
    ctx->ws_bytes = want;
    return GBS_OK;
}

int gbs_aux_ensure(gbs_ctx *ctx, size_t bytes, size_t keep) {
    if (bytes <= ctx->aux_bytes) return GBS_OK;
    GBS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    void *nb = nullptr;
    if (cudaMalloc(&nb, bytes) != cudaSuccess) {
        cudaGetLastError();
        return gbs_fail(ctx, GBS_E_NOMEM, "cannot allocate %zu bytes of auxiliary workspace", bytes);
    }
    if (keep && ctx->aux) {
        cudaError_t e = cudaMemcpyAsync(nb, ctx->aux, keep < ctx->aux_bytes ? keep : ctx->aux_bytes,
                                        cudaMemcpyDeviceToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) {
            cudaFree(nb);
            GBS_CUDA(ctx, e);
        }
    }
    if (ctx->aux) GBS_CUDA(ctx, cudaFree(ctx->aux));
    ctx->aux = nb;
    ctx->aux_bytes = bytes;
    return GBS_OK;
}

static int timing_fold_oldest(gbs_ctx *ctx) {
    const int R = gbs_ctx::kTimingRing;
    cudaEvent_t *e = ctx->tev + 2 * (ctx->t_tail % R);
    GBS_CUDA(ctx, cudaEventSynchronize(e[1]));
    float ms = 0.f;
    GBS_CUDA(ctx, cudaEventElapsedTime(&ms, e[0], e[1]));
    ctx->t_ms += ms;
    ctx->t_launches += 1;
    ctx->t_tail += 1;
    return GBS_OK;
}

int gbs_timing_begin(gbs_ctx *ctx) {
    if (!ctx->timing) return GBS_OK;
    if (ctx->t_head - ctx->t_tail == gbs_ctx::kTimingRing) {
        int st = timing_fold_oldest(ctx);
        if (st) return st;
    }
    GBS_CUDA(ctx, cudaEventRecord(ctx->tev[2 * (ctx->t_head % gbs_ctx::kTimingRing)], ctx->stream));
    return GBS_OK;
}

int gbs_timing_end(gbs_ctx *ctx) {
    if (!ctx->timing) return GBS_OK;
    GBS_CUDA(ctx, cudaEventRecord(ctx->tev[2 * (ctx->t_head % gbs_ctx::kTimingRing) + 1], ctx->stream));
    ctx->t_head += 1;
    return GBS_OK;
}

extern "C" {

int gbs_version(void) { return 100; }

int gbs_timing_enable(gbs_ctx *ctx, int enable) {
    if (!ctx) return GBS_E_INVALID;
    GBS_CUDA(ctx, cudaSetDevice(ctx->device));
    if (enable && !ctx->tev) {
        ctx->tev = new cudaEvent_t[2 * gbs_ctx::kTimingRing];
        for (int i = 0; i < 2 * gbs_ctx::kTimingRing; ++i)
            GBS_CUDA(ctx, cudaEventCreate(&ctx->tev[i]));
    }
    ctx->timing = enable != 0;
    return GBS_OK;
}

int gbs_timing_read(gbs_ctx *ctx, int reset, double *sweep_ms, long long *sweep_launches) {
    if (!ctx) return GBS_E_INVALID;
    GBS_CUDA(ctx, cudaSetDevice(ctx->device));
    while (ctx->tev && ctx->t_tail < ctx->t_head) {
        int st = timing_fold_oldest(ctx);
        if (st) return st;
    }
    if (sweep_ms) *sweep_ms = ctx->t_ms;
    if (sweep_launches) *sweep_launches = ctx->t_launches;
    if (reset) {
        ctx->t_ms = 0.0;
        ctx->t_launches = 0;
    }
    return GBS_OK;
}

int gbs_create(gbs_ctx **out, int device, void *cuda_stream) {
    if (!out) return GBS_E_INVALID;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return GBS_E_INVALID;
    }
    gbs_ctx *ctx = new gbs_ctx();
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMallocHost(&ctx->pinned, 4096) != cudaSuccess ||
        cudaMalloc(&ctx->dscratch, 256) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return GBS_E_CUDA;
    }
    *out = ctx;
    return GBS_OK;
}

int gbs_destroy(gbs_ctx *ctx) {
    if (!ctx) return GBS_E_INVALID;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->host_io) cudaFree(ctx->host_io);
    if (ctx->aux) cudaFree(ctx->aux);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    if (ctx->dscratch) cudaFree(ctx->dscratch);
    if (ctx->tev) {
        for (int i = 0; i < 2 * gbs_ctx::kTimingRing; ++i) cudaEventDestroy(ctx->tev[i]);
        delete[] ctx->tev;
    }
    delete ctx;
    return GBS_OK;
}

int gbs_set_stream(gbs_ctx *ctx, void *cuda_stream) {
    if (!ctx) return GBS_E_INVALID;
    ctx->stream = (cudaStream_t)cuda_stream;
    return GBS_OK;
}

const char *gbs_last_error(const gbs_ctx *ctx) { return ctx ? ctx->err : "null context"; }

int gbs_reserve(gbs_ctx *ctx, int n_pat, int n_max) {
    if (!ctx || n_pat < 0 || n_max < 0 || n_max > 40)
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_reserve: bad n_pat %d / n_max %d", n_pat, n_max);
    GBS_CUDA(ctx, cudaSetDevice(ctx->device));
    long long units = 0;
    size_t bytes = 0;
    for (int prec : {GBS_FP64, GBS_FP32_SPLIT, GBS_DD, GBS_FX, GBS_FX192}) {
        const long long u = sweep_units_upper_bound(n_pat, n_max, prec, sweep_split_of(ctx, prec));
        const size_t by = sweep_workspace_bytes_prec(n_pat, u, prec);
        if (u > units) units = u;
        if (by > bytes) bytes = by;
    }
    int st = gbs_ws_ensure(ctx, bytes);
    if (st) return st;
    // GBS_AUTO's rerun buffers
    const size_t aux = sweep_auto_bytes(n_pat);
    if (aux > ctx->aux_bytes) {
        GBS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (ctx->aux) GBS_CUDA(ctx, cudaFree(ctx->aux));
        ctx->aux = nullptr;
        ctx->aux_bytes = 0;
        if (cudaMalloc(&ctx->aux, aux) != cudaSuccess) {
            cudaGetLastError();
            return gbs_fail(ctx, GBS_E_NOMEM, "gbs_reserve: %zu bytes", aux);
        }
        ctx->aux_bytes = aux;
    }
    ctx->reserved = true;
    ctx->cap_pat = n_pat;
    ctx->cap_units = units;
    return GBS_OK;
}

int gbs_click_distribution(gbs_ctx *ctx, int M, const double *O, const double *logdet_sigmaQ, double *logp,
                           double *kappa) {
    if (!ctx) return GBS_E_INVALID;
    if (!O || !logdet_sigmaQ || !logp)
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_click_distribution: null pointer");
    GBS_CUDA(ctx, cudaSetDevice(ctx->device));
    return click_distribution(ctx, M, O, logdet_sigmaQ, logp, kappa);
}

int gbs_approx_sector_curves(gbs_ctx *ctx, int M, const double *O, const double *logdet_sigmaQ,
                             const uint64_t *pattern, int n, int order, int precision, int K, double *curves,
                             double *logP, int32_t *status) {
    if (!ctx) return GBS_E_INVALID;
    if (!O || !logdet_sigmaQ || !pattern || !curves || !logP || !status)
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_approx_sector_curves: null pointer");
    if (M < 1 || M > 128) return gbs_fail(ctx, GBS_E_INVALID, "gbs_approx_sector_curves: M = %d", M);
    GBS_CUDA(ctx, cudaSetDevice(ctx->device));
    return approx_sector_curves(ctx, M, O, logdet_sigmaQ, pattern, n, order, precision, K, curves, logP, status);
}

int gbs_sector_distribution(gbs_ctx *ctx, int M, const double *O, const double *logdet_sigmaQ, int L, double rho,
                            int K, int even_only, int precision, double *pkn) {
    if (!ctx) return GBS_E_INVALID;
    if (!O || !logdet_sigmaQ || !pkn) return gbs_fail(ctx, GBS_E_INVALID, "gbs_sector_distribution: null pointer");
    GBS_CUDA(ctx, cudaSetDevice(ctx->device));
    return sector_distribution(ctx, M, O, logdet_sigmaQ, L, rho, K, even_only, precision, pkn);
}

int gbs_autotune(gbs_ctx *ctx, int M, const double *O, const double *logdet_sigmaQ,
                 const uint64_t *patterns, int n_pat, int precision, int *best_split, double *best_ms) {
    if (!ctx) return GBS_E_INVALID;
    if (M < 1 || M > 128 || n_pat < 1 || !O || !logdet_sigmaQ || !patterns ||
        (precision != GBS_FP64 && precision != GBS_FP32_SPLIT && precision != GBS_DD && precision != GBS_FX))
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_autotune: bad arguments (M=%d, n_pat=%d, precision=%d)", M,
                        n_pat, precision);
    GBS_CUDA(ctx, cudaSetDevice(ctx->device));
    double *lp = nullptr;
    int32_t *st = nullptr;
    GBS_CUDA(ctx, cudaMalloc(&lp, sizeof(double) * (size_t)n_pat));
    if (cudaMalloc(&st, sizeof(int32_t) * (size_t)n_pat) != cudaSuccess) {
        cudaFree(lp);
        return gbs_fail(ctx, GBS_E_NOMEM, "gbs_autotune: cannot allocate %d statuses", n_pat);
    }
    int32_t *hst = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_pat);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int code = GBS_OK, best = -1;
    float best_t = 0.0f;
    const int saved = ctx->sweep_split[precision];
    const bool timing = ctx->timing;
    ctx->timing = false;
    if (!hst || cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        code = gbs_fail(ctx, GBS_E_NOMEM, "gbs_autotune: setup failed");
    } else {
        for (int s = 0; s <= 3 && code == GBS_OK; ++s) {
            ctx->sweep_split[precision] = s;
            code = sweep_exact(ctx, M, O, logdet_sigmaQ, patterns, n_pat, precision, lp, nullptr, nullptr, st);
            if (code) break;
            cudaEventRecord(e0, ctx->stream);
            for (int rep = 0; rep < 2 && code == GBS_OK; ++rep)
                code = sweep_exact(ctx, M, O, logdet_sigmaQ, patterns, n_pat, precision, lp, nullptr, nullptr, st);
            if (code) break;
            cudaEventRecord(e1, ctx->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess ||
                cudaMemcpy(hst, st, sizeof(int32_t) * (size_t)n_pat, cudaMemcpyDeviceToHost) != cudaSuccess) {
                code = gbs_fail(ctx, GBS_E_CUDA, "gbs_autotune: timing failed");
                break;
            }
            bool fits = true;  // a reservation too small for this split reports GBS_E_NOMEM
            for (int p = 0; p < n_pat; ++p) fits = fits && hst[p] != GBS_E_NOMEM;
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (fits && (best < 0 || ms < best_t)) {
                best = s;
                best_t = ms;
            }
        }
    }
    ctx->sweep_split[precision] = code == GBS_OK && best >= 0 ? best : saved;
    ctx->timing = timing;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    free(hst);
    cudaFree(lp);
    cudaFree(st);
    if (code) return code;
    if (best < 0) return gbs_fail(ctx, GBS_E_NOMEM, "gbs_autotune: no split fits the reserved workspace");
    if (best_split) *best_split = best;
    if (best_ms) *best_ms = best_t / 2.0;
    return GBS_OK;
}

int gbs_build_state(gbs_ctx *ctx, int M, const double *U, const double *r, double eta,
                    double *sigma, double *O, double *logdet_sigmaQ, int32_t *status_dev) {
    if (!ctx) return GBS_E_INVALID;
    if (M < 1 || M > 128 || !U || !r || !O || !logdet_sigmaQ || !(eta > 0.0) || eta > 1.0)
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_build_state: bad arguments (M=%d, eta=%g)", M, eta);
    GBS_CUDA(ctx, cudaSetDevice(ctx->device));
    return launch_build_state(ctx, M, U, r, eta, sigma, O, logdet_sigmaQ, status_dev);
}

int gbs_prob(gbs_ctx *ctx, int M, const double *O, const double *logdet_sigmaQ,
             const uint64_t *patterns, int n_pat, int order, int precision, double *logP,
             double *kappa, double *err_bound, int32_t *status) {
    if (!ctx) return GBS_E_INVALID;
    if (M < 1 || M > 128 || n_pat < 0 || !O || !logdet_sigmaQ || (n_pat && (!patterns || !logP)))
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_prob: bad arguments (M=%d, n_pat=%d)", M, n_pat);
    if (precision != GBS_FP64 && precision != GBS_FP32_SPLIT && precision != GBS_DD && precision != GBS_FX &&
        precision != GBS_FF && precision != GBS_AUTO && precision != GBS_FX192)
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_prob: unknown precision %d", precision);
    if (order == 0 && precision == GBS_FF)
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_prob: float-float serves the approximation (order > 0) only");
    if (order > 0 && precision == GBS_FX192)
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_prob: 192-bit fixed point serves the exact sum (order 0) only");
    if (n_pat == 0) return GBS_OK;
    GBS_CUDA(ctx, cudaSetDevice(ctx->device));
    if (order == 0 && precision == GBS_AUTO)
        return sweep_auto(ctx, M, O, logdet_sigmaQ, patterns, n_pat, logP, kappa, err_bound, status);
    if (order == 0)
        return sweep_exact(ctx, M, O, logdet_sigmaQ, patterns, n_pat, precision, logP, kappa,
                           err_bound, status);
    return approx_prob(ctx, M, O, logdet_sigmaQ, patterns, n_pat, order, precision == GBS_AUTO ? GBS_FF : precision,
                       logP, kappa, err_bound, status);
}

int gbs_prob_partial(gbs_ctx *ctx, int M, const double *O, const uint64_t *patterns, int n_pat, int precision,
                     int part, int nparts, double *partial, int32_t *pflag) {
    if (!ctx) return GBS_E_INVALID;
    if (M < 1 || M > 128 || n_pat < 0 || !O || (n_pat && (!patterns || !partial || !pflag)) || nparts < 1 ||
        nparts > 65536 || part < 0 || part >= nparts)
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_prob_partial: bad arguments (M=%d, n_pat=%d, part %d of %d)", M,
                        n_pat, part, nparts);
    if (precision != GBS_FP64 && precision != GBS_FP32_SPLIT && precision != GBS_DD && precision != GBS_FX)
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_prob_partial: precision %d (FP64, FP32 split, DD or FX)", precision);
    if (n_pat == 0) return GBS_OK;
    GBS_CUDA(ctx, cudaSetDevice(ctx->device));
    return sweep_slice(ctx, M, O, patterns, n_pat, precision, part, nparts, partial, pflag);
}

int gbs_prob_combine(gbs_ctx *ctx, const double *logdet_sigmaQ, const uint64_t *patterns, int n_pat, int precision,
                     int nparts, const double *partials, const int32_t *pflags, double *logP, double *kappa,
                     double *err_bound, int32_t *status) {
    if (!ctx) return GBS_E_INVALID;
    if (n_pat < 0 || !logdet_sigmaQ || nparts < 1 || nparts > 65536 ||
        (n_pat && (!patterns || !partials || !pflags || !logP)))
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_prob_combine: bad arguments (n_pat=%d, nparts=%d)", n_pat, nparts);
    if (precision != GBS_FP64 && precision != GBS_FP32_SPLIT && precision != GBS_DD && precision != GBS_FX)
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_prob_combine: precision %d (FP64, FP32 split, DD or FX)", precision);
    if (n_pat == 0) return GBS_OK;
    GBS_CUDA(ctx, cudaSetDevice(ctx->device));
    return sweep_combine(ctx, logdet_sigmaQ, patterns, n_pat, precision, nparts, partials, pflags, logP, kappa,
                         err_bound, status);
}

int gbs_run_host(gbs_ctx *ctx, int M, const double *U_host, const double *r_host, double eta,
                 const uint64_t *patterns_host, int n_pat, int order, int precision,
                 double *logP_host, double *kappa_host, double *err_host, int32_t *status_host) {
    if (!ctx) return GBS_E_INVALID;
    if (M < 1 || M > 128 || n_pat < 0 || !U_host || !r_host || (n_pat && (!patterns_host || !logP_host)))
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_run_host: bad arguments");
    GBS_CUDA(ctx, cudaSetDevice(ctx->device));
    size_t N = 2 * (size_t)M;
    // device layout: U | r | O | logdet | status | patterns | logP | kappa | err | pstatus
    size_t off_U = 0, off_r = off_U + 2 * M * M * 8, off_O = off_r + M * 8,
           off_ld = off_O + N * N * 8, off_st = off_ld + 8, off_pat = off_st + 8,
           off_lp = off_pat + (size_t)n_pat * 16, off_k = off_lp + (size_t)n_pat * 8,
           off_e = off_k + (size_t)n_pat * 8, off_ps = off_e + (size_t)n_pat * 8,
           total = off_ps + (size_t)n_pat * 4 + 256;
    if (total > ctx->host_io_bytes) {
        GBS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (ctx->host_io) GBS_CUDA(ctx, cudaFree(ctx->host_io));
        ctx->host_io = nullptr;
        ctx->host_io_bytes = 0;
        if (cudaMalloc(&ctx->host_io, total) != cudaSuccess) {
            cudaGetLastError();
            return gbs_fail(ctx, GBS_E_NOMEM, "gbs_run_host: cannot allocate %zu bytes", total);
        }
        ctx->host_io_bytes = total;
    }
    char *b = (char *)ctx->host_io;
    cudaStream_t s = ctx->stream;
    GBS_CUDA(ctx, cudaMemcpyAsync(b + off_U, U_host, 2 * M * M * 8, cudaMemcpyHostToDevice, s));
    GBS_CUDA(ctx, cudaMemcpyAsync(b + off_r, r_host, M * 8, cudaMemcpyHostToDevice, s));
    if (n_pat)
        GBS_CUDA(ctx, cudaMemcpyAsync(b + off_pat, patterns_host, (size_t)n_pat * 16,
                                      cudaMemcpyHostToDevice, s));
    int st = launch_build_state(ctx, M, (double *)(b + off_U), (double *)(b + off_r), eta, nullptr,
                                (double *)(b + off_O), (double *)(b + off_ld),
                                (int32_t *)(b + off_st));
    if (st) return st;
    st = gbs_prob(ctx, M, (double *)(b + off_O), (double *)(b + off_ld), (uint64_t *)(b + off_pat),
                  n_pat, order, precision, (double *)(b + off_lp), (double *)(b + off_k),
                  (double *)(b + off_e), (int32_t *)(b + off_ps));
    if (st) return st;
    int32_t state_status = 0;
    GBS_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, b + off_st, 4, cudaMemcpyDeviceToHost, s));
    if (n_pat) {
        GBS_CUDA(ctx, cudaMemcpyAsync(logP_host, b + off_lp, n_pat * 8, cudaMemcpyDeviceToHost, s));
        if (kappa_host)
            GBS_CUDA(ctx, cudaMemcpyAsync(kappa_host, b + off_k, n_pat * 8, cudaMemcpyDeviceToHost, s));
        if (err_host)
            GBS_CUDA(ctx, cudaMemcpyAsync(err_host, b + off_e, n_pat * 8, cudaMemcpyDeviceToHost, s));
        if (status_host)
            GBS_CUDA(ctx, cudaMemcpyAsync(status_host, b + off_ps, n_pat * 4, cudaMemcpyDeviceToHost, s));
    }
    GBS_CUDA(ctx, cudaStreamSynchronize(s));
    memcpy(&state_status, ctx->pinned, 4);
    if (state_status)
        return gbs_fail(ctx, state_status, "gbs_run_host: state build rejected the inputs");
    return GBS_OK;
}

int gbs_grad(gbs_ctx *ctx, int M, const double *O, const double *logdet_sigmaQ,
             const uint64_t *patterns, int n_pat, const double *w, double *dsigmaQ, double *logP,
             int32_t *status) {
    if (!ctx) return GBS_E_INVALID;
    if (M < 1 || M > 128 || n_pat < 1 || !O || !logdet_sigmaQ || !patterns || !w || !dsigmaQ)
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_grad: bad arguments (M=%d, n_pat=%d)", M, n_pat);
    GBS_CUDA(ctx, cudaSetDevice(ctx->device));
    return grad_sigmaQ(ctx, M, O, logdet_sigmaQ, patterns, n_pat, w, dsigmaQ, logP, status);
}

int gbs_grad_approx(gbs_ctx *ctx, int M, const double *O, const double *logdet_sigmaQ,
                    const uint64_t *patterns, int n_pat, int order, const double *w, double *dsigmaQ,
                    double *logP, int32_t *status) {
    if (!ctx) return GBS_E_INVALID;
    if (M < 1 || M > 128 || n_pat < 1 || !O || !logdet_sigmaQ || !patterns || !w || !dsigmaQ)
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_grad_approx: bad arguments (M=%d, n_pat=%d)", M, n_pat);
    GBS_CUDA(ctx, cudaSetDevice(ctx->device));
    return approx_grad(ctx, M, O, logdet_sigmaQ, patterns, n_pat, order, w, dsigmaQ, logP, status);
}

int gbs_grad_params(gbs_ctx *ctx, int M, const double *U, const double *r, double eta,
                    const double *dsigmaQ, double *dU, double *dr, double *deta) {
    if (!ctx) return GBS_E_INVALID;
    if (M < 1 || M > 128 || !U || !r || !dsigmaQ || !dU || !dr || !deta || !(eta > 0.0) || eta > 1.0)
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_grad_params: bad arguments");
    GBS_CUDA(ctx, cudaSetDevice(ctx->device));
    return grad_params(ctx, M, U, r, eta, dsigmaQ, dU, dr, deta);
}

int gbs_clements_unitary(gbs_ctx *ctx, int M, const double *theta, const double *phi, double *U) {
    if (!ctx) return GBS_E_INVALID;
    if (M < 2 || M > 128 || !theta || !phi || !U)
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_clements_unitary: bad arguments");
    GBS_CUDA(ctx, cudaSetDevice(ctx->device));
    return clements_unitary(ctx, M, theta, phi, U);
}

int gbs_clements_grad(gbs_ctx *ctx, int M, const double *theta, const double *phi, const double *U,
                      const double *dU, double *dtheta, double *dphi) {
    if (!ctx) return GBS_E_INVALID;
    if (M < 2 || M > 128 || !theta || !phi || !U || !dU || !dtheta || !dphi)
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_clements_grad: bad arguments");
    GBS_CUDA(ctx, cudaSetDevice(ctx->device));
    return clements_grad(ctx, M, theta, phi, U, dU, dtheta, dphi);
}

int gbs_gen_patterns(gbs_ctx *ctx, uint64_t seed, uint32_t stream, int M, int n_lo, int n_hi,
                     int n_pat, uint64_t *out) {
    if (!ctx) return GBS_E_INVALID;
    if (M < 1 || M > 128 || n_lo < 0 || n_hi < n_lo || n_hi > M || n_pat < 0 || (n_pat && !out))
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_gen_patterns: bad arguments");
    if (n_pat == 0) return GBS_OK;
    GBS_CUDA(ctx, cudaSetDevice(ctx->device));
    return launch_gen_patterns(ctx, seed, stream, M, n_lo, n_hi, n_pat, out);
}

int gbs_set_pair_from(gbs_ctx *ctx, int n_min) {
    if (!ctx) return GBS_E_INVALID;
    if (n_min < 3 || n_min > 80)
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_set_pair_from: %d outside [3, 80]", n_min);
    ctx->pair_from = n_min;
    return GBS_OK;
}

int gbs_peak_flops(gbs_ctx *ctx, int kind, double *flops) {
    if (!ctx || !flops || kind < 0 || kind > 4) return GBS_E_INVALID;
    GBS_CUDA(ctx, cudaSetDevice(ctx->device));
    return peak_flops(ctx, kind, flops);
}

}  // extern "C"
