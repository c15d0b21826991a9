// Gradients of L = sum_p w_p log P_p (not in the paper; the state-build adjoint
// lets squeezing, loss and the interferometer be fitted to click data).
//
// From log P = -1/2 log det sigma_Q + log T(A_S), A = sigma_Q^{-1} and
// d det(A_Z)^{-1/2} = -1/2 det(A_Z)^{-1/2} tr(A_Z^{-1} dA_Z):
//     dT = tr(Gbar dA_S),  Gbar = sum_Z (-1)^{n-|Z|} (-1/2) tau_Z A_Z^{-1},
//     dL/dsigma_Q = -1/2 (sum_p w_p) A - A H A,   H = sum_p (w_p / T_p) embed(Gbar_p).
// Gbar and T cancel together by the condition number kappa of the signed sum
// (1e14..1e19 on improbable patterns), so every subset Cholesky, inverse and
// sum is double-double; after the division by T the result is an ordinary
// FP64 number.  One warp per subset; chunks of subsets per CTA; chunk partials
// summed per pattern in order (deterministic).
//
// Then the chain through sigma_Q = eta R diag(d) R^T + (1 - eta/2) I (R the xp
// form of U, d = e^{-2r}/2 on x, e^{2r}/2 on p) and through the rectangular
// mesh U = T_last ... T_1, T(theta, phi) = [[e^{i phi} cos, -sin], [e^{i phi} sin, cos]].
#include "dd.cuh"
#include "gbs_internal.cuh"

namespace {

constexpr int kGradMaxN = 16;            // clicks per pattern on the gradient path
constexpr int kGD = 2 * kGradMaxN;       // largest subset matrix (32 x 32)
constexpr int kGradWarps = 2;            // warps per CTA
constexpr int kChunkLog = 11;            // 2048 subsets per CTA

struct GradWarpSmem {
    dd L[kGD * kGD];     // Cholesky factor (lower)
    dd X[kGD * kGD];     // columns of A_Z^{-1}
    dd acc[kGD * kGD];   // this warp's share of Gbar (2n x 2n, S-local rows 2a + alpha)
};

__global__ void __launch_bounds__(32 * kGradWarps) grad_subsets_kernel(
    int M, const double *__restrict__ O, const uint64_t *__restrict__ pats, int n_pat,
    const long long *__restrict__ chunk_off, double *__restrict__ part_hi, double *__restrict__ part_lo,
    double *__restrict__ part_T, int *__restrict__ flags) {
    extern __shared__ __align__(16) unsigned char gsm[];
    GradWarpSmem *ws = (GradWarpSmem *)gsm;
    __shared__ int modes[128];
    __shared__ int s_n, s_p;
    __shared__ double s_T[kGradWarps][2];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long cid = blockIdx.x;
    if (threadIdx.x == 0) {
        int lo = 0, hi = n_pat;
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (chunk_off[mid] <= cid) lo = mid; else hi = mid;
        }
        int p = lo;
        while (p + 1 < n_pat && chunk_off[p + 1] <= cid) ++p;
        s_p = p;
        int n = 0;
        for (int i = 0; i < M; ++i) {
            uint64_t w = i < 64 ? pats[2 * p] : pats[2 * p + 1];
            if (w >> (i & 63) & 1ull) modes[n++] = i;
        }
        s_n = n;
    }
    __syncthreads();
    const int p = s_p, n = s_n, D = 2 * n, N2 = 2 * M;
    const long long chunk = cid - chunk_off[p];
    GradWarpSmem &S = ws[wid];
    for (int f = lane; f < D * D; f += 32) S.acc[f] = dd(0.0);
    dd tsum = dd(0.0);
    bool bad = false;
    const long long z0 = chunk << kChunkLog;
    long long z1 = z0 + (1ll << kChunkLog);
    if (z1 > (1ll << n)) z1 = 1ll << n;
    __syncwarp();
    for (long long z = z0 + wid; z < z1; z += kGradWarps) {
        const int k = __popcll((unsigned long long)z), d = 2 * k;
        // the lane's row: mode (i/2)-th set bit of z, quadrature i & 1
        int gi = 0, li = 0;
        if (lane < d) {
            int c = lane >> 1, a = 0;
            for (; a < n; ++a)
                if (z >> a & 1) { if (c == 0) break; --c; }
            gi = modes[a] + (lane & 1) * M;
            li = 2 * a + (lane & 1);
        }
        // lower triangle of A_Z = (I - O)_Z, exact in double-double
        for (int j = 0; j < d; ++j) {
            int gj = __shfl_sync(0xffffffffu, gi, j);
            if (lane < d && lane >= j) S.L[lane * kGD + j] = dd_two_sum(lane == j ? 1.0 : 0.0, -O[(size_t)gi * N2 + gj]);
        }
        __syncwarp();
        // left-looking Cholesky, lane = row
        for (int j = 0; j < d; ++j) {
            if (lane == j) {
                dd s = S.L[j * kGD + j];
                for (int m = 0; m < j; ++m) s = s - S.L[j * kGD + m] * S.L[j * kGD + m];
                if (!(s.hi > 0.0)) bad = true;
                // sqrt by one Newton step from the double root
                double x = sqrt(s.hi);
                dd r = s - dd(x) * dd(x);
                S.L[j * kGD + j] = dd_two_sum(x, r.hi / (2.0 * x));
            }
            __syncwarp();
            if (lane > j && lane < d) {
                dd s = S.L[lane * kGD + j];
                for (int m = 0; m < j; ++m) s = s - S.L[lane * kGD + m] * S.L[j * kGD + m];
                S.L[lane * kGD + j] = s / S.L[j * kGD + j];
            }
            __syncwarp();
        }
        // tau = prod 1/L_ii; sign (-1)^{n - k}
        dd tau = dd(1.0);
        for (int i = 0; i < d; ++i) tau = tau / S.L[i * kGD + i];
        if ((n - k) & 1) tau = -tau;
        tsum += tau;
        // column `lane` of A_Z^{-1}: L y = e_lane, L^T x = y
        if (lane < d) {
            const int j = lane;
            for (int i = 0; i < j; ++i) S.X[i * kGD + j] = dd(0.0);
            S.X[j * kGD + j] = dd(1.0) / S.L[j * kGD + j];
            for (int i = j + 1; i < d; ++i) {
                dd s = dd(0.0);
                for (int m = j; m < i; ++m) s += S.L[i * kGD + m] * S.X[m * kGD + j];
                S.X[i * kGD + j] = -(s / S.L[i * kGD + i]);
            }
            for (int i = d - 1; i >= 0; --i) {
                dd s = S.X[i * kGD + j];
                for (int m = i + 1; m < d; ++m) s = s - S.L[m * kGD + i] * S.X[m * kGD + j];
                S.X[i * kGD + j] = s / S.L[i * kGD + i];
            }
        }
        __syncwarp();
        // acc[loc_i][loc_j] += (-1/2) (+-tau) (A_Z^{-1})_{ij}; lanes own distinct columns
        const dd c = tau * dd(-0.5);
        for (int i = 0; i < d; ++i) {
            int lr = __shfl_sync(0xffffffffu, li, i);
            if (lane < d) S.acc[lr * D + li] += c * S.X[i * kGD + lane];
        }
        __syncwarp();
    }
    if (lane == 0) {
        s_T[wid][0] = tsum.hi;
        s_T[wid][1] = tsum.lo;
        if (bad) atomicOr(flags + p, 1);
    }
    if (bad) atomicOr(flags + p, 1);
    __syncthreads();
    // sum the warps' shares (fixed order) and write the chunk partial
    const size_t base = (size_t)cid * kGD * kGD;
    for (int f = threadIdx.x; f < D * D; f += 32 * kGradWarps) {
        dd s = ws[0].acc[f];
        for (int w = 1; w < kGradWarps; ++w) s += ws[w].acc[f];
        part_hi[base + f] = s.hi;
        part_lo[base + f] = s.lo;
    }
    if (threadIdx.x == 0) {
        dd t = dd(s_T[0][0], s_T[0][1]);
        for (int w = 1; w < kGradWarps; ++w) t += dd(s_T[w][0], s_T[w][1]);
        part_T[2 * cid] = t.hi;
        part_T[2 * cid + 1] = t.lo;
    }
}

// per pattern: sum the chunk partials in order, F_p = (w_p / T_p) Gbar_p, log P_p
__global__ void grad_finalize_kernel(int M, const uint64_t *__restrict__ pats, int n_pat,
                                     const long long *__restrict__ chunk_off,
                                     const double *__restrict__ part_hi, const double *__restrict__ part_lo,
                                     const double *__restrict__ part_T, const double *__restrict__ w,
                                     const double *__restrict__ logdet, double *__restrict__ F,
                                     double *__restrict__ logP, int32_t *__restrict__ status,
                                     const int *__restrict__ flags) {
    const int p = blockIdx.x;
    __shared__ double s_scale;
    __shared__ int s_n;
    if (threadIdx.x == 0) {
        int n = __popcll(pats[2 * p]) + __popcll(pats[2 * p + 1]);
        s_n = n;
        dd T = dd(0.0);
        for (long long c = chunk_off[p]; c < chunk_off[p + 1]; ++c) T += dd(part_T[2 * c], part_T[2 * c + 1]);
        int st = flags[p] ? GBS_E_NOT_SPD : (T.hi > 0.0 ? GBS_OK : GBS_E_NONPOSITIVE);
        if (status) status[p] = st;
        if (logP) logP[p] = st ? nan("") : -0.5 * (*logdet) + log(T.hi) + log1p(T.lo / T.hi);
        s_scale = st ? 0.0 : w[p] / (T.hi + T.lo);
    }
    __syncthreads();
    const int D = 2 * s_n;
    for (int f = threadIdx.x; f < D * D; f += blockDim.x) {
        dd s = dd(0.0);
        for (long long c = chunk_off[p]; c < chunk_off[p + 1]; ++c)
            s += dd(part_hi[(size_t)c * kGD * kGD + f], part_lo[(size_t)c * kGD * kGD + f]);
        F[(size_t)p * kGD * kGD + f] = (s.hi + s.lo) * s_scale;
    }
}

// H[i][j] = sum_p F_p at the rows of S_p (patterns in order: deterministic); sumw
__global__ void grad_scatter_kernel(int M, const uint64_t *__restrict__ pats, int n_pat,
                                    const double *__restrict__ F, const double *__restrict__ w,
                                    double *__restrict__ H, double *__restrict__ sumw) {
    const int N = 2 * M;
    const int i = blockIdx.y * blockDim.y + threadIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && j == 0) {
        double s = 0.0;
        for (int p = 0; p < n_pat; ++p) s += w[p];
        *sumw = s;
    }
    if (i >= N || j >= N) return;
    const int mi = i < M ? i : i - M, ai = i < M ? 0 : 1;
    const int mj = j < M ? j : j - M, aj = j < M ? 0 : 1;
    double h = 0.0;
    for (int p = 0; p < n_pat; ++p) {
        const uint64_t lo = pats[2 * p], hi = pats[2 * p + 1];
        auto has = [&](int m) { return ((m < 64 ? lo >> m : hi >> (m - 64)) & 1ull) != 0; };
        if (!has(mi) || !has(mj)) continue;
        // S-local index = rank of the mode among the clicked ones
        auto rank = [&](int m) {
            int r = __popcll(lo & (m >= 64 ? ~0ull : ((1ull << m) - 1)));
            if (m >= 64) r += __popcll(hi & ((1ull << (m - 64)) - 1));
            return r;
        };
        const int n = __popcll(lo) + __popcll(hi);
        const int D = 2 * n;
        h += F[(size_t)p * kGD * kGD + (2 * rank(mi) + ai) * D + (2 * rank(mj) + aj)];
    }
    H[(size_t)i * N + j] = h;
}

// C = X Y for N x N row-major matrices, with X, Y = I - O when the flag says so
__global__ void grad_matmul_kernel(int N, const double *__restrict__ X, int x_is_A,
                                   const double *__restrict__ Y, int y_is_A, double *__restrict__ C) {
    const int i = blockIdx.y * blockDim.y + threadIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N || j >= N) return;
    double s = 0.0;
    for (int k = 0; k < N; ++k) {
        double x = X[(size_t)i * N + k], y = Y[(size_t)k * N + j];
        if (x_is_A) x = (i == k ? 1.0 : 0.0) - x;
        if (y_is_A) y = (k == j ? 1.0 : 0.0) - y;
        s = fma(x, y, s);
    }
    C[(size_t)i * N + j] = s;
}

// dsigma_Q = -1/2 sumw A - AHA   (AHA precomputed)
__global__ void grad_sigma_kernel(int N, const double *__restrict__ O, const double *__restrict__ AHA,
                                  const double *__restrict__ sumw, double *__restrict__ dsq) {
    const int i = blockIdx.y * blockDim.y + threadIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N || j >= N) return;
    const double a = (i == j ? 1.0 : 0.0) - O[(size_t)i * N + j];
    dsq[(size_t)i * N + j] = -0.5 * (*sumw) * a - AHA[(size_t)i * N + j];
}

// chain: dR = 2 eta W R diag(d), dr_j, deta (W the symmetrised dsigma_Q)
__device__ __forceinline__ double R_of(const double *U, int M, int i, int j) {
    int ui = i < M ? i : i - M, uj = j < M ? j : j - M;
    double re = U[2 * (ui * M + uj)], im = U[2 * (ui * M + uj) + 1];
    if (i < M) return j < M ? re : -im;
    return j < M ? im : re;
}

// WR = W R with W = (dsq + dsq^T)/2
__global__ void grad_wr_kernel(int M, const double *__restrict__ U, const double *__restrict__ dsq,
                               double *__restrict__ WR) {
    const int N = 2 * M;
    const int i = blockIdx.y * blockDim.y + threadIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N || j >= N) return;
    double s = 0.0;
    for (int k = 0; k < N; ++k) s += 0.5 * (dsq[(size_t)i * N + k] + dsq[(size_t)k * N + i]) * R_of(U, M, k, j);
    WR[(size_t)i * N + j] = s;
}

__global__ void grad_params_kernel(int M, const double *__restrict__ U, const double *__restrict__ r,
                                   double eta, const double *__restrict__ dsq, const double *__restrict__ pw,
                                   double *__restrict__ dU, double *__restrict__ dr, double *__restrict__ deta) {
    const int N = 2 * M;
    auto dvec = [&](int j) { int m = j < M ? j : j - M; return 0.5 * exp(j < M ? -2.0 * r[m] : 2.0 * r[m]); };
    // dU from dR = 2 eta (W R) diag(d)
    for (int f = threadIdx.x; f < M * M; f += blockDim.x) {
        int i = f / M, j = f - i * M;
        double dr_ij = 2 * eta * pw[i * N + j] * dvec(j), dr_iMjM = 2 * eta * pw[(i + M) * N + j + M] * dvec(j + M);
        double dr_ijM = 2 * eta * pw[i * N + j + M] * dvec(j + M), dr_iMj = 2 * eta * pw[(i + M) * N + j] * dvec(j);
        dU[2 * f] = dr_ij + dr_iMjM;
        dU[2 * f + 1] = -dr_ijM + dr_iMj;
    }
    // (R^T W R)_jj = sum_k R_kj (W R)_kj
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        double qx = 0.0, qp = 0.0;
        for (int k = 0; k < N; ++k) {
            qx += R_of(U, M, k, j) * pw[k * N + j];
            qp += R_of(U, M, k, j + M) * pw[k * N + j + M];
        }
        dr[j] = eta * (-2.0 * dvec(j) * qx + 2.0 * dvec(j + M) * qp);
    }
    if (threadIdx.x == 0) {
        double s = 0.0, trw = 0.0;
        for (int j = 0; j < N; ++j) {
            double q = 0.0;
            for (int k = 0; k < N; ++k) q += R_of(U, M, k, j) * pw[k * N + j];
            s += dvec(j) * q;
            trw += dsq[(size_t)j * N + j];
        }
        *deta = s - 0.5 * trw;
    }
}

// the rectangular mesh: cell order of layer l = pairs (m, m+1) with m of the parity of l
__device__ __forceinline__ int cell_mode(int M, int c) {
    int per2 = M - 1;  // cells in two consecutive layers (M/2 + (M-1)/2 ... for any M)
    int layer = 0, base = 0;
    for (;;) {
        int cnt = (M - 1 - (layer & 1) + 1) / 2;  // m = parity, parity+2, ... < M - 1
        if (c < base + cnt) return (layer & 1) + 2 * (c - base);
        base += cnt;
        ++layer;
    }
    (void)per2;
}

__global__ void clements_unitary_kernel(int M, const double *__restrict__ theta, const double *__restrict__ phi,
                                        double *__restrict__ U) {
    const int col = threadIdx.x;
    const int ncell = M * (M - 1) / 2;
    for (int f = col; f < M * M; f += blockDim.x) {
        U[2 * f] = (f / M == f % M) ? 1.0 : 0.0;
        U[2 * f + 1] = 0.0;
    }
    __syncthreads();
    for (int c = 0; c < ncell; ++c) {
        const int m = cell_mode(M, c);
        double st, ct, sp, cp;
        sincos(theta[c], &st, &ct);
        sincos(phi[c], &sp, &cp);
        if (col < M) {
            double ar = U[2 * (m * M + col)], ai = U[2 * (m * M + col) + 1];
            double br = U[2 * ((m + 1) * M + col)], bi = U[2 * ((m + 1) * M + col) + 1];
            double ear = cp * ar - sp * ai, eai = cp * ai + sp * ar;  // e^{i phi} a
            U[2 * (m * M + col)] = ct * ear - st * br;
            U[2 * (m * M + col) + 1] = ct * eai - st * bi;
            U[2 * ((m + 1) * M + col)] = st * ear + ct * br;
            U[2 * ((m + 1) * M + col) + 1] = st * eai + ct * bi;
        }
        __syncthreads();
    }
}

// reverse pass through the mesh: the cell inputs are recovered from its outputs
// (T is unitary), so no forward storage is needed
__global__ void clements_grad_kernel(int M, const double *__restrict__ theta, const double *__restrict__ phi,
                                     const double *__restrict__ Ufinal, const double *__restrict__ dU,
                                     double *__restrict__ dtheta, double *__restrict__ dphi) {
    extern __shared__ double cs[];   // U (2 M M) | G (2 M M) | reduction (2 * blockDim)
    double *Uc = cs, *G = cs + 2 * M * M, *red = cs + 4 * M * M;
    const int col = threadIdx.x;
    const int ncell = M * (M - 1) / 2;
    for (int f = col; f < 2 * M * M; f += blockDim.x) {
        Uc[f] = Ufinal[f];
        G[f] = dU[f];
    }
    __syncthreads();
    for (int c = ncell - 1; c >= 0; --c) {
        const int m = cell_mode(M, c);
        double st, ct, sp, cp;
        sincos(theta[c], &st, &ct);
        sincos(phi[c], &sp, &cp);
        double gth = 0.0, gph = 0.0;
        if (col < M) {
            const double o0r = Uc[2 * (m * M + col)], o0i = Uc[2 * (m * M + col) + 1];
            const double o1r = Uc[2 * ((m + 1) * M + col)], o1i = Uc[2 * ((m + 1) * M + col) + 1];
            // inputs: e a = ct o0 + st o1, b = -st o0 + ct o1
            const double ear = ct * o0r + st * o1r, eai = ct * o0i + st * o1i;
            const double br = -st * o0r + ct * o1r, bi = -st * o0i + ct * o1i;
            const double ar = cp * ear + sp * eai, ai = cp * eai - sp * ear;   // a = e^{-i phi} (e a)
            const double g0r = G[2 * (m * M + col)], g0i = G[2 * (m * M + col) + 1];
            const double g1r = G[2 * ((m + 1) * M + col)], g1i = G[2 * ((m + 1) * M + col) + 1];
            // do0/dtheta = -st (e a) - ct b, do1/dtheta = ct (e a) - st b
            const double d0r = -st * ear - ct * br, d0i = -st * eai - ct * bi;
            const double d1r = ct * ear - st * br, d1i = ct * eai - st * bi;
            gth = g0r * d0r + g0i * d0i + g1r * d1r + g1i * d1i;
            // do0/dphi = i ct (e a), do1/dphi = i st (e a)
            gph = g0r * (-ct * eai) + g0i * (ct * ear) + g1r * (-st * eai) + g1i * (st * ear);
            // adjoint inputs: G_a = e^{-i phi} (ct g0 + st g1), G_b = -st g0 + ct g1
            const double hr = ct * g0r + st * g1r, hi = ct * g0i + st * g1i;
            G[2 * (m * M + col)] = cp * hr + sp * hi;
            G[2 * (m * M + col) + 1] = cp * hi - sp * hr;
            G[2 * ((m + 1) * M + col)] = -st * g0r + ct * g1r;
            G[2 * ((m + 1) * M + col) + 1] = -st * g0i + ct * g1i;
            Uc[2 * (m * M + col)] = ar;
            Uc[2 * (m * M + col) + 1] = ai;
            Uc[2 * ((m + 1) * M + col)] = br;
            Uc[2 * ((m + 1) * M + col) + 1] = bi;
        }
        red[col] = gth;
        red[blockDim.x + col] = gph;
        __syncthreads();
        if (col == 0) {
            double a = 0.0, b = 0.0;
            for (int q = 0; q < M; ++q) { a += red[q]; b += red[blockDim.x + q]; }
            dtheta[c] = a;
            dphi[c] = b;
        }
        __syncthreads();
    }
}

__global__ void grad_plan_kernel(const uint64_t *__restrict__ pats, int n_pat, int M,
                                 long long *__restrict__ chunk_off, int *__restrict__ flags) {
    if (threadIdx.x || blockIdx.x) return;
    long long run = 0;
    for (int p = 0; p < n_pat; ++p) {
        chunk_off[p] = run;
        int n = __popcll(pats[2 * p]) + __popcll(pats[2 * p + 1]);
        run += n > kChunkLog ? (1ll << (n - kChunkLog)) : 1;
        flags[p] = 0;
    }
    chunk_off[n_pat] = run;
}

size_t al(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

int grad_sigmaQ(gbs_ctx *ctx, int M, const double *O, const double *logdet, const uint64_t *pats,
                int n_pat, const double *w, double *dsq, double *logP, int32_t *status) {
    // every pattern must be valid and have at most kGradMaxN clicks: checked on the host
    // from a copy of the pattern words (one small readback)
    size_t pb = (size_t)n_pat * 16;
    uint64_t *hp = (uint64_t *)malloc(pb + 16);
    if (!hp) return gbs_fail(ctx, GBS_E_NOMEM, "gbs_grad: host buffer");
    GBS_CUDA(ctx, cudaMemcpyAsync(hp, pats, pb, cudaMemcpyDeviceToHost, ctx->stream));
    GBS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    long long chunks = 0;
    for (int p = 0; p < n_pat; ++p) {
        uint64_t lo = hp[2 * p], hi = hp[2 * p + 1];
        int n = __builtin_popcountll(lo) + __builtin_popcountll(hi);
        bool out_of_range = (M < 64 && (lo >> M)) || (M <= 64 && hi) || (M > 64 && M < 128 && (hi >> (M - 64)));
        if (n > kGradMaxN || out_of_range) {
            free(hp);
            return gbs_fail(ctx, GBS_E_INVALID, "gbs_grad: pattern %d has %d clicks (at most %d) or a detector >= M",
                            p, n, kGradMaxN);
        }
        chunks += n > kChunkLog ? (1ll << (n - kChunkLog)) : 1;
    }
    free(hp);
    const int N = 2 * M;
    size_t o_off = 0, o_flags = al(o_off + 8 * ((size_t)n_pat + 1)), o_phi = al(o_flags + 4 * (size_t)n_pat),
           o_plo = al(o_phi + 8 * (size_t)chunks * kGD * kGD), o_pT = al(o_plo + 8 * (size_t)chunks * kGD * kGD),
           o_F = al(o_pT + 16 * (size_t)chunks), o_H = al(o_F + 8 * (size_t)n_pat * kGD * kGD),
           o_T1 = al(o_H + 8 * (size_t)N * N), o_T2 = al(o_T1 + 8 * (size_t)N * N), o_sw = al(o_T2 + 8 * (size_t)N * N),
           total = o_sw + 64;
    int st = gbs_ws_ensure(ctx, total);
    if (st) return st;
    char *b = (char *)ctx->ws;
    long long *chunk_off = (long long *)(b + o_off);
    int *flags = (int *)(b + o_flags);
    double *phi_ = (double *)(b + o_phi), *plo = (double *)(b + o_plo), *pT = (double *)(b + o_pT);
    double *F = (double *)(b + o_F), *H = (double *)(b + o_H), *T1 = (double *)(b + o_T1),
           *T2 = (double *)(b + o_T2), *sw = (double *)(b + o_sw);
    grad_plan_kernel<<<1, 32, 0, ctx->stream>>>(pats, n_pat, M, chunk_off, flags);
    GBS_CUDA(ctx, cudaGetLastError());
    const size_t smem = sizeof(GradWarpSmem) * kGradWarps;
    GBS_CUDA(ctx, cudaFuncSetAttribute(grad_subsets_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    st = gbs_timing_begin(ctx);
    if (st) return st;
    grad_subsets_kernel<<<(unsigned)chunks, 32 * kGradWarps, smem, ctx->stream>>>(M, O, pats, n_pat, chunk_off,
                                                                                   phi_, plo, pT, flags);
    GBS_CUDA(ctx, cudaGetLastError());
    st = gbs_timing_end(ctx);
    if (st) return st;
    grad_finalize_kernel<<<n_pat, 256, 0, ctx->stream>>>(M, pats, n_pat, chunk_off, phi_, plo, pT, w, logdet, F,
                                                         logP, status, flags);
    GBS_CUDA(ctx, cudaGetLastError());
    dim3 blk(16, 16), grd((N + 15) / 16, (N + 15) / 16);
    grad_scatter_kernel<<<grd, blk, 0, ctx->stream>>>(M, pats, n_pat, F, w, H, sw);
    grad_matmul_kernel<<<grd, blk, 0, ctx->stream>>>(N, H, 0, O, 1, T1);    // H A
    grad_matmul_kernel<<<grd, blk, 0, ctx->stream>>>(N, O, 1, T1, 0, T2);   // A (H A)
    grad_sigma_kernel<<<grd, blk, 0, ctx->stream>>>(N, O, T2, sw, dsq);
    GBS_CUDA(ctx, cudaGetLastError());
    return GBS_OK;
}

int grad_params(gbs_ctx *ctx, int M, const double *U, const double *r, double eta, const double *dsq,
                double *dU, double *dr, double *deta) {
    const int N = 2 * M;
    int st = gbs_ws_ensure(ctx, sizeof(double) * (size_t)N * N);
    if (st) return st;
    double *WR = (double *)ctx->ws;
    dim3 blk(16, 16), grd((N + 15) / 16, (N + 15) / 16);
    grad_wr_kernel<<<grd, blk, 0, ctx->stream>>>(M, U, dsq, WR);
    grad_params_kernel<<<1, 256, 0, ctx->stream>>>(M, U, r, eta, dsq, WR, dU, dr, deta);
    GBS_CUDA(ctx, cudaGetLastError());
    return GBS_OK;
}

int clements_unitary(gbs_ctx *ctx, int M, const double *theta, const double *phi, double *U) {
    clements_unitary_kernel<<<1, 128, 0, ctx->stream>>>(M, theta, phi, U);
    GBS_CUDA(ctx, cudaGetLastError());
    return GBS_OK;
}

int clements_grad(gbs_ctx *ctx, int M, const double *theta, const double *phi, const double *U,
                  const double *dU, double *dtheta, double *dphi) {
    const int threads = 128;
    const size_t smem = sizeof(double) * (4 * (size_t)M * M + 2 * threads);
    GBS_CUDA(ctx, cudaFuncSetAttribute(clements_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    clements_grad_kernel<<<1, threads, smem, ctx->stream>>>(M, theta, phi, U, dU, dtheta, dphi);
    GBS_CUDA(ctx, cudaGetLastError());
    return GBS_OK;
}
