// Synthetic click patterns from the counter-based generator Philox4x32-10
// (Salmon, Moraes, Dror, Shaw, SC'11): one thread per pattern.  The stream of
// words and the Fisher-Yates draw are specified in gbs.h; the host generator
// in the test inputs implements the same definition, bit for bit.
#include "gbs_internal.cuh"

namespace {

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
#pragma unroll
    for (int rnd = 0; rnd < 10; ++rnd) {
        if (rnd) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
        uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
        uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

struct WordStream {
    uint32_t buf[4];
    uint32_t idx, blk, stream, k0, k1;
    int pos;
    __device__ uint32_t next() {
        if (pos == 4) {
            buf[0] = idx;
            buf[1] = blk++;
            buf[2] = stream;
            buf[3] = 0;
            philox4x32_10(buf, k0, k1);
            pos = 0;
        }
        return buf[pos++];
    }
};

__device__ __forceinline__ uint32_t range32(uint32_t w, uint32_t span) {
    return (uint32_t)(((uint64_t)w * (uint64_t)span) >> 32);
}

__global__ void gen_patterns_kernel(uint64_t seed, uint32_t stream, int M, int n_lo, int n_hi,
                                    int n_pat, uint64_t *__restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pat) return;
    WordStream ws;
    ws.idx = (uint32_t)i;
    ws.blk = 0;
    ws.stream = stream;
    ws.k0 = (uint32_t)(seed & 0xFFFFFFFFu);
    ws.k1 = (uint32_t)(seed >> 32);
    ws.pos = 4;
    uint8_t perm[128];
    for (int k = 0; k < M; ++k) perm[k] = (uint8_t)k;
    int n = n_lo + (int)range32(ws.next(), (uint32_t)(n_hi - n_lo + 1));
    uint64_t lo = 0, hi = 0;
    for (int k = 0; k < n; ++k) {
        int j = k + (int)range32(ws.next(), (uint32_t)(M - k));
        uint8_t t = perm[k];
        perm[k] = perm[j];
        perm[j] = t;
        int m = perm[k];
        if (m < 64) lo |= 1ull << m;
        else hi |= 1ull << (m - 64);
    }
    out[2 * i] = lo;
    out[2 * i + 1] = hi;
}

}  // namespace

int launch_gen_patterns(gbs_ctx *ctx, uint64_t seed, uint32_t stream, int M, int n_lo, int n_hi,
                        int n_pat, uint64_t *out) {
    int threads = 128, blocks = (n_pat + threads - 1) / threads;
    gen_patterns_kernel<<<blocks, threads, 0, ctx->stream>>>(seed, stream, M, n_lo, n_hi, n_pat, out);
    GBS_CUDA(ctx, cudaGetLastError());
    return GBS_OK;
}
