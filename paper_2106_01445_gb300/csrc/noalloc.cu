// gbs_prob_noalloc: the exact signed subset sweep without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs while a stream is being
// captured into someone else's CUDA graph, processes whose device memory is
// entirely held by another framework's caching pool, and latency-critical
// serving loops that must never wait on the allocator.  gbs_prob sizes a
// context-owned workspace with cudaMalloc; this entry point instead keeps the
// sweep's scratch (pattern plan and per-unit partial sums) in one fixed array
// in the library's own device memory, declared below.  Every GPU that loads the
// library holds that array until the process exits.
#include <mutex>

#include "gbs_internal.cuh"

namespace {

// 8 MiB: up to 16384 patterns and ~3.3e5 work units per call.
constexpr size_t kNoAllocBytes = size_t(8) << 20;
constexpr int kNoAllocMaxPatterns = 16384;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_mu;
void *g_addr[kMaxDevices] = {nullptr};

// The host-side symbol is only a stand-in; the device address of the array is
// looked up once per device, with that device current.
int scratch_address(gbs_ctx *ctx, void **out) {
    if (ctx->device < 0 || ctx->device >= kMaxDevices)
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_prob_noalloc: device %d out of range", ctx->device);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[ctx->device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return gbs_fail(ctx, GBS_E_CUDA, "gbs_prob_noalloc: cudaGetSymbolAddress failed: %s",
                            cudaGetErrorString(e));
        g_addr[ctx->device] = p;
    }
    *out = g_addr[ctx->device];
    return GBS_OK;
}

}  // namespace

extern "C" int gbs_prob_noalloc(gbs_ctx *ctx, int M, const double *O, const double *logdet_sigmaQ,
                                const uint64_t *patterns, int n_pat, int n_max, int precision,
                                double *logP, double *kappa, double *err_bound, int32_t *status) {
    if (!ctx) return GBS_E_INVALID;
    if (M < 1 || M > 128 || n_pat < 0 || n_max < 0 || n_max > 40 || !O || !logdet_sigmaQ ||
        (n_pat && (!patterns || !logP)))
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_prob_noalloc: bad arguments (M=%d, n_pat=%d, n_max=%d)",
                        M, n_pat, n_max);
    if (precision != GBS_FP64 && precision != GBS_FP32_SPLIT && precision != GBS_DD && precision != GBS_FX)
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_prob_noalloc: unknown precision %d", precision);
    if (n_pat > kNoAllocMaxPatterns)
        return gbs_fail(ctx, GBS_E_INVALID,
                        "gbs_prob_noalloc: %d patterns exceed the fixed scratch limit of %d", n_pat,
                        kNoAllocMaxPatterns);
    const long long units = sweep_units_upper_bound(n_pat, n_max, precision, sweep_split_of(ctx, precision));
    const size_t need = sweep_workspace_bytes(n_pat, units);
    if (need > kNoAllocBytes)
        return gbs_fail(ctx, GBS_E_INVALID,
                        "gbs_prob_noalloc: %d patterns of up to %d clicks need %zu bytes of scratch, "
                        "more than the fixed %zu", n_pat, n_max, need, kNoAllocBytes);
    if (n_pat == 0) return GBS_OK;
    GBS_CUDA(ctx, cudaSetDevice(ctx->device));
    void *scratch = nullptr;
    int st = scratch_address(ctx, &scratch);
    if (st) return st;
    return sweep_exact_on(ctx, scratch, kNoAllocBytes, M, O, logdet_sigmaQ, patterns, n_pat,
                          precision, logP, kappa, err_bound, status);
}
