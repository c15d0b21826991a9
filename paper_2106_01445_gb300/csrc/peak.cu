// Pipe-peak microbenchmarks: FP32 and FP64 FMA throughput of the whole GPU,
// register-resident, eight independent dependency chains per thread; and the
// throughput of the fused Schur-update entry c - w0 b0 - w1 b1 in double-double and
// in 128-bit fixed point, four independent chains per thread with loop-carried
// operands.  Used as the denominators of the arithmetic roofline of the subset sweep.
#include "dd.cuh"
#include "fx.cuh"
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

__global__ void dd_update_loop(double *out, int iters) {
    dd c0(0.5 + threadIdx.x * 1e-6, 1e-20), c1(0.25, 1e-21), c2(0.125, 0.0), c3(0.0625, 0.0);
    const dd w0(0.3, 1e-18), w1(0.1, 3e-19);
    for (int it = 0; it < iters; ++it) {
        const dd n0 = dd_fms2(c0, c1, c2, c3, w0);
        const dd n1 = dd_fms2(c1, c2, c3, c0, w1);
        const dd n2 = dd_fms2(c2, c3, c0, c1, w0);
        const dd n3 = dd_fms2(c3, c0, c1, c2, w1);
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    const double s = (c0.hi + c1.hi) + (c2.hi + c3.hi);
    if (s == -12345.678) out[0] = s;
}

// the sweep's own fixed-point update entry, the symmetric form c + t_i + t_j -
// (u'_i0 u'_j0 + u'_i1 u'_j1) with two unsigned truncated products (fx_sym_update)
__global__ void fx_update_loop(double *out, int iters) {
    fx c0 = fx_from_double(0.5 + threadIdx.x * 1e-6), c1 = fx_from_double(0.25);
    fx c2 = fx_from_double(1.125), c3 = fx_from_double(0.0625);
    const fx w0 = fx_from_double(1.3), w1 = fx_from_double(2.1), t0 = fx_from_double(-0.5);
    for (int it = 0; it < iters; ++it) {
        const fx n0 = fx_sym_update(c0, c1, c2, t0, c3, w0, t0);
        const fx n1 = fx_sym_update(c1, c2, c3, t0, c0, w1, t0);
        const fx n2 = fx_sym_update(c2, c3, c0, t0, c1, w0, t0);
        const fx n3 = fx_sym_update(c3, c0, c1, t0, c2, w1, t0);
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    const uint32_t s = c0.w[0] ^ c1.w[1] ^ c2.w[2] ^ c3.w[3];
    if (s == 0x9e3779b9u) out[0] = 1.0;
}

// 32-bit integer multiply-add throughput (IMAD), eight independent chains per thread:
// the issue rate of the pipe that carries the fixed-point products
__global__ void imad_loop(unsigned *out, int iters, unsigned a, unsigned b) {
    unsigned x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
    unsigned x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
            x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
        }
    }
    const unsigned s = ((x0 ^ x1) + (x2 ^ x3)) ^ ((x4 + x5) ^ (x6 + x7));
    if (s == 0x12345u) out[0] = s;
}

}  // namespace

int peak_flops(gbs_ctx *ctx, int kind, double *flops) {
    int threads = 256, blocks = ctx->num_sms * 8;
    const int iters = kind == 0 ? 4096 : kind == 1 ? 128 : kind == 2 ? 128 : kind == 3 ? 1024 : 4096;
    cudaEvent_t e0, e1;
    GBS_CUDA(ctx, cudaEventCreate(&e0));
    GBS_CUDA(ctx, cudaEventCreate(&e1));
    float best = 1e30f;
    for (int rep = 0; rep < 5; ++rep) {
        GBS_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
        if (kind == 0)
            fma_loop<float><<<blocks, threads, 0, ctx->stream>>>((float *)ctx->dscratch, iters,
                                                                 0.999999f, 1e-7f);
        else if (kind == 1)
            fma_loop<double><<<blocks, threads, 0, ctx->stream>>>((double *)ctx->dscratch, iters,
                                                                  0.999999, 1e-7);
        else if (kind == 2)
            dd_update_loop<<<blocks, threads, 0, ctx->stream>>>((double *)ctx->dscratch, iters);
        else if (kind == 3)
            fx_update_loop<<<blocks, threads, 0, ctx->stream>>>((double *)ctx->dscratch, iters);
        else
            imad_loop<<<blocks, threads, 0, ctx->stream>>>((unsigned *)ctx->dscratch, iters, 2654435761u,
                                                          12345u);
        GBS_CUDA(ctx, cudaGetLastError());
        GBS_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
        GBS_CUDA(ctx, cudaEventSynchronize(e1));
        float ms = 0;
        GBS_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
        if (rep && ms < best) best = ms;  // first launch is warm-up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // FMA loops: 8 chains x 16 FMA x 2 flops; update loops: 4 entries x 4 flops; the IMAD
    // loop counts one per multiply-add (8 chains x 16)
    const double per = kind <= 1 ? 2.0 * 8 * 16 : kind == 4 ? 8.0 * 16 : 4.0 * 4;
    double fl = per * (double)iters * threads * blocks;
    *flops = fl / (best * 1e-3);
    return GBS_OK;
}
