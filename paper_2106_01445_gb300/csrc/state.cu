// State build: sigma, O = I - sigma_Q^{-1} and log det sigma_Q of the lossy
// Gaussian output state (Methods, "Model"; "Partition function" normalisation).
//
// Uniform loss commutes with the interferometer, so with the orthogonal
// xp-form R of U,
//     sigma   = R diag(s) R^T,         s = eta sigma_in + (1 - eta)/2,
//     sigma_Q = R diag(s + 1/2) R^T,   sigma_Q^{-1} = R diag(1/(s + 1/2)) R^T,
//     log det sigma_Q = sum_j log1p(eta (2 - eta) sinh^2 r_j).
// Every entry is an independent length-2M dot product: no factorisation, one
// thread per entry, the whole GPU in one launch.
#include "gbs_internal.cuh"

namespace {

__device__ __forceinline__ double R_entry(const double *U, int M, int i, int j) {
    // R = [[Re U, -Im U], [Im U, Re U]] in xp order
    int ui = i < M ? i : i - M, uj = j < M ? j : j - M;
    double re = U[2 * (ui * M + uj)], im = U[2 * (ui * M + uj) + 1];
    if (i < M) return j < M ? re : -im;
    return j < M ? im : re;
}

__global__ void state_kernel(int M, const double *__restrict__ U, const double *__restrict__ r,
                             double eta, double *__restrict__ sigma, double *__restrict__ O,
                             double *__restrict__ logdet, int32_t *__restrict__ status) {
    const int N = 2 * M;
    int i = blockIdx.y * blockDim.y + threadIdx.y;
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N && k < N) {
        double acc_s = 0.0, acc_a = 0.0;
        for (int j = 0; j < N; ++j) {
            int jm = j < M ? j : j - M;
            double rj = r[jm];
            // x quadratures get e^{-2r}/2, p quadratures e^{2r}/2
            double sin_ = 0.5 * exp(j < M ? -2.0 * rj : 2.0 * rj);
            double s = eta * sin_ + 0.5 * (1.0 - eta);
            double prod = R_entry(U, M, i, j) * R_entry(U, M, k, j);
            acc_s = fma(prod, s, acc_s);
            acc_a = fma(prod, 1.0 / (s + 0.5), acc_a);
        }
        if (sigma) sigma[i * N + k] = acc_s;
        O[i * N + k] = (i == k ? 1.0 : 0.0) - acc_a;
        // unitarity residual |U^dag U - 1| on the M x M block
        if (i < M && k < M) {
            double re = 0.0, im = 0.0;
            for (int j = 0; j < M; ++j) {
                double ar = U[2 * (j * M + i)], ai = -U[2 * (j * M + i) + 1];
                double br = U[2 * (j * M + k)], bi = U[2 * (j * M + k) + 1];
                re += ar * br - ai * bi;
                im += ar * bi + ai * br;
            }
            re -= (i == k) ? 1.0 : 0.0;
            if (!(fabs(re) <= 1e-10 && fabs(im) <= 1e-10)) atomicExch(status, (int32_t)GBS_E_INVALID);
        }
    }
    const int lin = threadIdx.y * blockDim.x + threadIdx.x;  // whole warp 0 of block (0, 0)
    if (blockIdx.x == 0 && blockIdx.y == 0 && lin < 32) {
        double acc = 0.0;
        for (int j = lin; j < M; j += 32) {
            double rj = r[j];
            if (!(rj >= 0.0) || !isfinite(rj)) atomicExch(status, (int32_t)GBS_E_INVALID);
            double sh = sinh(rj);
            acc += log1p(eta * (2.0 - eta) * sh * sh);
        }
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lin == 0) *logdet = acc;
    }
}

}  // namespace

int launch_build_state(gbs_ctx *ctx, int M, const double *U, const double *r, double eta,
                       double *sigma, double *O, double *logdet, int32_t *status_dev) {
    int32_t *st = status_dev ? status_dev : ctx->dscratch;
    GBS_CUDA(ctx, cudaMemsetAsync(st, 0, sizeof(int32_t), ctx->stream));
    int N = 2 * M;
    dim3 blk(16, 16), grd((N + 15) / 16, (N + 15) / 16);
    state_kernel<<<grd, blk, 0, ctx->stream>>>(M, U, r, eta, sigma, O, logdet, st);
    GBS_CUDA(ctx, cudaGetLastError());
    if (status_dev) return GBS_OK;
    GBS_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, st, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    GBS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    int32_t h = *(int32_t *)ctx->pinned;
    if (h) return gbs_fail(ctx, h, "gbs_build_state: U not unitary to 1e-10, or r < 0 / not finite");
    return GBS_OK;
}
