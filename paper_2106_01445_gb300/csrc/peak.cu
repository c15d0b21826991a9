// Pipe-peak microbenchmark: FP32 and FP64 FMA throughput of the whole GPU,
// register-resident, eight independent dependency chains per thread.  Used as
// the denominator of the arithmetic roofline of the subset sweep.
#include "gbs_internal.cuh"

namespace {

template <typename T>
__global__ void fma_loop(T *out, int iters, T a, T b) {
    T x0 = threadIdx.x * (T)1e-3, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
    T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
            x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
        }
    }
    T s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
    if (s == (T)-12345.678) out[0] = s;  // keeps the loop alive
}

}  // namespace

int peak_flops(gbs_ctx *ctx, int kind, double *flops) {
    int threads = 256, blocks = ctx->num_sms * 8;
    int iters = kind == 0 ? 4096 : 128;
    cudaEvent_t e0, e1;
    GBS_CUDA(ctx, cudaEventCreate(&e0));
    GBS_CUDA(ctx, cudaEventCreate(&e1));
    float best = 1e30f;
    for (int rep = 0; rep < 5; ++rep) {
        GBS_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
        if (kind == 0)
            fma_loop<float><<<blocks, threads, 0, ctx->stream>>>((float *)ctx->dscratch, iters,
                                                                 0.999999f, 1e-7f);
        else
            fma_loop<double><<<blocks, threads, 0, ctx->stream>>>((double *)ctx->dscratch, iters,
                                                                  0.999999, 1e-7);
        GBS_CUDA(ctx, cudaGetLastError());
        GBS_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
        GBS_CUDA(ctx, cudaEventSynchronize(e1));
        float ms = 0;
        GBS_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
        if (rep && ms < best) best = ms;  // first launch is warm-up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    double fl = 2.0 * 8 * 16 * (double)iters * threads * blocks;
    *flops = fl / (best * 1e-3);
    return GBS_OK;
}
