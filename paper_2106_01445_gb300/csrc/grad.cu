// Gradients of L = sum_p w_p log P_p (not in the paper; the state-build adjoint
// lets squeezing, loss and the interferometer be fitted to click data).
//
// From log P = -1/2 log det sigma_Q + log T(A_S), A = sigma_Q^{-1} and
// d det(A_Z)^{-1/2} = -1/2 det(A_Z)^{-1/2} tr(A_Z^{-1} dA_Z):
//     dT = tr(Gbar dA_S),  Gbar = sum_Z (-1)^{n-|Z|} (-1/2) tau_Z A_Z^{-1},
//     dL/dsigma_Q = -1/2 (sum_p w_p) A - A H A,   H = sum_p (w_p / T_p) embed(Gbar_p).
// Gbar and T cancel together by the condition number kappa of the signed sum
// (1e14..1e19 on improbable patterns), so the whole computation is double-double;
// after the division by T the result is an ordinary FP64 number.  Gbar = dT/dA_S is
// computed in reverse mode through the same include/exclude Schur recursion that
// evaluates T (O(2^n) work instead of a factorisation and inverse per subset); one
// CTA per pattern, its units in order (deterministic).
//
// Then the chain through sigma_Q = eta R diag(d) R^T + (1 - eta/2) I (R the xp
// form of U, d = e^{-2r}/2 on x, e^{2r}/2 on p) and through the rectangular
// mesh U = T_last ... T_1, T(theta, phi) = [[e^{i phi} cos, -sin], [e^{i phi} sin, cos]].
#include "dd.cuh"
#include "gbs_internal.cuh"

namespace {

constexpr int kGradMaxN = 24;            // clicks per pattern on the gradient path
constexpr int kGD = 2 * kGradMaxN;       // largest pattern matrix (48 x 48)
constexpr int kTM = 7;                   // modes of a unit's subtree (2^7 leaves)
constexpr int kTreeThreads = 128;

__host__ __device__ constexpr int gsym(int d) { return d * (d + 1) / 2; }
// packed upper-triangle index of (i, j), i <= j
__host__ __device__ constexpr int gpidx(int d, int i, int j) { return i * d - (i * (i - 1)) / 2 + (j - i); }
__device__ __forceinline__ int gpany(int d, int i, int j) { return i <= j ? gpidx(d, i, j) : gpidx(d, j, i); }
// level l of a unit's subtree: 2^l nodes of dimension 2 (kTM - l), packed, back to back
__host__ __device__ constexpr int lvl_off(int l) {
    int s = 0;
    for (int q = 0; q < l; ++q) s += (1 << q) * gsym(2 * (kTM - q));
    return s;
}
constexpr int lvl_cap() {
    int m = 0;
    for (int l = 0; l < kTM; ++l) m = (1 << l) * gsym(2 * (kTM - l)) > m ? (1 << l) * gsym(2 * (kTM - l)) : m;
    return m;
}
constexpr int y_cap() {
    int m = 2 * (kGD - 2);
    for (int l = 0; l < kTM; ++l) m = (1 << l) * 4 * (kTM - l - 1) > m ? (1 << l) * 4 * (kTM - l - 1) : m;
    return m;
}
constexpr int kNodes = (1 << kTM) - 1;   // nodes of levels 0..kTM-1
// shared memory (double-double elements)
constexpr int kChunkBits = 8;           // a chunk: at most 2^8 units sharing their high prefix modes
constexpr int kUD = 2 * (kChunkBits + kTM);  // largest unit matrix (low prefix modes + subtree)
// SM: the chunk's matrix (included high prefix modes, every low prefix mode, the subtree
// modes), then its adjoint Gs; UM, Gf: one unit's matrix and adjoint; Gam: the adjoint of
// SM's trailing block after the high pivots, summed over the chunk's units
constexpr int kOffSM = 0, kOffGs = gsym(kGD), kOffUM = 2 * gsym(kGD), kOffGf = kOffUM + gsym(kUD),
              kOffGam = kOffGf + gsym(kUD), kOffLv = kOffGam + gsym(kUD);
constexpr int kOffAdjA = kOffLv + lvl_off(kTM), kOffAdjB = kOffAdjA + lvl_cap();
constexpr int kOffQ = kOffAdjB + lvl_cap(), kOffRs = kOffQ + 3 * kNodes, kOffS = kOffRs + kNodes;
constexpr int kOffY = kOffS + kNodes, kOffPreQ = kOffY + y_cap(), kOffPreRs = kOffPreQ + 3 * kGradMaxN;
constexpr int kOffHiQ = kOffPreRs + kGradMaxN, kOffHiRs = kOffHiQ + 3 * kGradMaxN;
constexpr int kTreeSmem = kOffHiRs + kGradMaxN;

// (i, j), i <= j, of packed entry f of an even dimension d: rows p and d - 1 - p folded
__device__ __forceinline__ void fold_ij(int f, int d, int &i, int &j) {
    const int w = d + 1, p = f / w, k = f - p * w;
    if (k < d - p) {
        i = p;
        j = p + k;
    } else {
        i = d - 1 - p;
        j = i + (k - (d - p));
    }
}

// One 2x2 pivot of the packed D x D unit matrix, eliminated by the CTA: rows and
// columns >= c0 + 2 receive C - W B^T (W = B P^{-1}); the pivot rows stay as they were
// (the reverse pass reads them).  Returns det^{-1/2}; stores P^{-1} and det^{-1/2}.
__device__ dd tree_pivot(dd *UM, int D, int c0, dd *Wb, dd *Qout, dd *rsout, int *bad) {
    const int t = threadIdx.x;
    const dd p00 = UM[gpidx(D, c0, c0)], p01 = UM[gpidx(D, c0, c0 + 1)], p11 = UM[gpidx(D, c0 + 1, c0 + 1)];
    const dd det = dd_dot2(p00, p11, -p01, p01);
    const dd rs = dd_rsqrt(det), inv = rs * rs;
    const dd q00 = p11 * inv, q01 = -p01 * inv, q11 = p00 * inv;
    if (t == 0) {
        Qout[0] = q00;
        Qout[1] = q01;
        Qout[2] = q11;
        *rsout = rs;
        if (!(det.hi > 0.0)) atomicOr(bad, 1);
    }
    const int Dt = D - c0 - 2;
    for (int i = t; i < Dt; i += kTreeThreads) {
        const dd b0 = UM[gpidx(D, c0, c0 + 2 + i)], b1 = UM[gpidx(D, c0 + 1, c0 + 2 + i)];
        Wb[2 * i] = dd_dot2(q00, b0, q01, b1);
        Wb[2 * i + 1] = dd_dot2(q01, b0, q11, b1);
    }
    __syncthreads();
    for (int f = t; f < gsym(Dt); f += kTreeThreads) {
        int i, j;
        fold_ij(f, Dt, i, j);
        dd &c = UM[gpidx(D, c0 + 2 + i, c0 + 2 + j)];
        c = dd_fms2(c, Wb[2 * i], UM[gpidx(D, c0, c0 + 2 + j)], Wb[2 * i + 1], UM[gpidx(D, c0 + 1, c0 + 2 + j)]);
    }
    __syncthreads();
    return rs;
}

// Back through the pivots e = np - 1 .. 0 of the packed D x D matrix Mx (pivot rows kept):
// G holds the adjoint of the trailing block below the last pivot; each pivot adds its rows,
// -rs Y with Y = P^{-1} B G, and its block, (Y B^T P^{-1})(i, j) - V P^{-1} / 2 (the
// prefactor's det^{-1/2}, V the value it multiplies).  Q: 3 entries of P^{-1} per pivot.
__device__ void reverse_pivots(const dd *Mx, dd *G, int D, int np, const dd *Qs, dd V, dd *Yb) {
    const int t = threadIdx.x;
    for (int e = np - 1; e >= 0; --e) {
        const int c0 = 2 * e, R = D - c0 - 2;
        const dd *Q = Qs + 3 * e;
        for (int j = t; j < R; j += kTreeThreads) {
            dd z0 = dd(0.0), z1 = dd(0.0);
            for (int i = 0; i < R; ++i) {
                const dd g = G[gpany(D, c0 + 2 + i, c0 + 2 + j)];
                z0 = z0 + Mx[gpidx(D, c0, c0 + 2 + i)] * g;
                z1 = z1 + Mx[gpidx(D, c0 + 1, c0 + 2 + i)] * g;
            }
            Yb[2 * j] = dd_dot2(Q[0], z0, Q[1], z1);
            Yb[2 * j + 1] = dd_dot2(Q[1], z0, Q[2], z1);
        }
        __syncthreads();
        for (int f = t; f < 2 * R + 3; f += kTreeThreads) {
            if (f < 2 * R) {
                const int a = f / R, j = f - a * R;
                G[gpidx(D, c0 + a, c0 + 2 + j)] = -Yb[2 * j + a];
            } else {
                const int i = (f - 2 * R) == 2 ? 1 : 0, j = (f - 2 * R) == 0 ? 0 : 1;
                dd yb0 = dd(0.0), yb1 = dd(0.0);
                for (int c = 0; c < R; ++c) {
                    const dd y = Yb[2 * c + i];
                    yb0 = yb0 + y * Mx[gpidx(D, c0, c0 + 2 + c)];
                    yb1 = yb1 + y * Mx[gpidx(D, c0 + 1, c0 + 2 + c)];
                }
                const dd qj0 = Q[j == 0 ? 0 : 1], qj1 = Q[j == 0 ? 1 : 2];
                G[gpidx(D, c0 + i, c0 + j)] = dd_dot2(yb0, qj0, yb1, qj1) - V * Q[i + j] * dd(0.5);
            }
        }
        __syncthreads();
    }
}

// Gbar_p = dT/dA_S by reverse mode through the include/exclude Schur recursion.
// Units = (pattern, include/exclude choice of the first q = n - m modes), m = min(n, 7).
// A unit's value V = (-1)^{q-k} tau_prefix S(root): its k included prefix modes are
// eliminated (pivot rows kept), then the subtree over the last m modes is expanded
// breadth first with every level kept, S(node) = rs S(include child) - S(exclude child)
// (S = 1 at a leaf).  Reverse, with Gamma(node) = dS(node)/dC_node:
//   rest block:  rs Gamma(inc) - Gamma(exc)
//   pivot rows:  -rs Y,  Y = P^{-1} B Gamma(inc)
//   pivot block: rs (Y B^T P^{-1} - S(inc) P^{-1} / 2)
// then back through the prefix pivots the same way (with -V P^{-1} / 2 from tau_prefix).
// One CTA per chunk: an aligned run of 2^b units of one pattern, whose first b prefix modes
// (the low ones) vary and the rest (the high ones) are fixed.  The chunk eliminates its
// included high modes once, from the matrix on its high, low and subtree rows (SM); each
// unit then takes SM's trailing block on its included low modes and the subtree, eliminates
// those, runs the subtree and its reverse, and adds its adjoint into the trailing block's
// (Gam); at the end Gam goes back through the high pivots once, with V = the chunk's sum
// (the adjoint of a shared step is linear in what flows into it), and the chunk's partial
// Gbar and T are written; the chunks of a pattern are summed in order afterwards.
__global__ void __launch_bounds__(kTreeThreads) grad_tree_kernel(int M, const double *__restrict__ O,
                                                               const uint64_t *__restrict__ pats, int n_pat,
                                                               const int *__restrict__ chunk_p,
                                                               const long long *__restrict__ chunk_u, size_t pst,
                                                               double *__restrict__ part_hi,
                                                               double *__restrict__ part_lo,
                                                               double *__restrict__ part_T, int *__restrict__ flags) {
    extern __shared__ __align__(16) unsigned char gsm[];
    dd *const base = (dd *)gsm;
    dd *const SM = base + kOffSM, *const Gs = base + kOffGs, *const UM = base + kOffUM, *const Gf = base + kOffGf;
    dd *const Gam = base + kOffGam, *const Lv = base + kOffLv;
    dd *const nQ = base + kOffQ, *const nrs = base + kOffRs, *const nS = base + kOffS, *const Yb = base + kOffY;
    dd *const preQ = base + kOffPreQ, *const prers = base + kOffPreRs;
    dd *const hiQ = base + kOffHiQ, *const hiRs = base + kOffHiRs;
    __shared__ int modes[128];
    __shared__ int smrow[kGD];   // row of SM -> pattern row (2 x detector index + x/p)
    __shared__ int umrow[kUD];   // row of a unit's matrix -> row of SM's trailing block
    __shared__ int s_n, s_kh, s_kl, s_bad;
    __shared__ dd s_T, s_V;
    const int t = threadIdx.x, ch = blockIdx.x, p = chunk_p[ch], N2 = 2 * M;
    const long long u_begin = chunk_u[2 * ch], u_end = chunk_u[2 * ch + 1];
    if (t == 0) {
        int n = 0;
        for (int i = 0; i < M; ++i) {
            const uint64_t w = i < 64 ? pats[2 * p] : pats[2 * p + 1];
            if (w >> (i & 63) & 1ull) modes[n++] = i;
        }
        s_n = n;
        s_bad = 0;
        s_T = dd(n == 0 && u_begin == 0 ? 1.0 : 0.0);
    }
    __syncthreads();
    const int n = s_n, m = n < kTM ? n : kTM, q = n - m, Dn = 2 * n;
    // the chunk's 2^bl units vary the prefix modes 0..bl-1; modes bl..q-1 are fixed by u_begin
    const int bl = u_end > u_begin ? 63 - __clzll(u_end - u_begin) : 0;
    const long long hi = u_begin >> bl;
    if (t == 0) {
        int r = 0;
        for (int a = bl; a < q; ++a)
            if (hi >> (a - bl) & 1) {
                smrow[r++] = 2 * a;
                smrow[r++] = 2 * a + 1;
            }
        s_kh = r / 2;
        for (int a = 0; a < bl; ++a) {
            smrow[r++] = 2 * a;
            smrow[r++] = 2 * a + 1;
        }
        for (int a = q; a < n; ++a) {
            smrow[r++] = 2 * a;
            smrow[r++] = 2 * a + 1;
        }
    }
    __syncthreads();
    const int kh = s_kh, Ds = 2 * (kh + bl + m), Dr = 2 * (bl + m);
    // the chunk's rows of A = I - O (exact in double-double), its high pivots, and a zero Gam
    for (int f = t; f < gsym(Ds); f += kTreeThreads) {
        int i, j;
        fold_ij(f, Ds, i, j);
        const int ri = smrow[i], rj = smrow[j];
        const int gi = modes[ri >> 1] + (ri & 1) * M, gj = modes[rj >> 1] + (rj & 1) * M;
        SM[gpidx(Ds, i, j)] = dd_two_sum(i == j ? 1.0 : 0.0, -O[(size_t)gi * N2 + gj]);
    }
    for (int f = t; f < gsym(Dr); f += kTreeThreads) Gam[f] = dd(0.0);
    __syncthreads();
    dd tau_h = dd(1.0);
    for (int e = 0; e < kh; ++e) tau_h = tau_h * tree_pivot(SM, Ds, 2 * e, Yb, hiQ + 3 * e, hiRs + e, &s_bad);
    for (long long u = u_begin; n > 0 && u < u_end; ++u) {
        const long long lb = u - u_begin;
        if (t == 0) {
            int r = 0;
            for (int a = 0; a < bl; ++a)
                if (lb >> a & 1) {
                    umrow[r++] = 2 * a;
                    umrow[r++] = 2 * a + 1;
                }
            s_kl = r / 2;
            for (int a = 0; a < m; ++a) {
                umrow[r++] = 2 * (bl + a);
                umrow[r++] = 2 * (bl + a) + 1;
            }
        }
        __syncthreads();
        const int kl = s_kl, k = kh + kl, D0 = 2 * (kl + m), o = 2 * kh;
        // the unit's matrix: SM's trailing block on its included low modes and the subtree
        for (int f = t; f < gsym(D0); f += kTreeThreads) {
            int i, j;
            fold_ij(f, D0, i, j);
            UM[gpidx(D0, i, j)] = SM[gpidx(Ds, o + umrow[i], o + umrow[j])];
        }
        __syncthreads();
        dd tau = tau_h;
        for (int e = 0; e < kl; ++e) tau = tau * tree_pivot(UM, D0, 2 * e, Yb, preQ + 3 * e, prers + e, &s_bad);
        // level 0 of the subtree: the trailing 2m x 2m block
        for (int f = t; f < gsym(2 * m); f += kTreeThreads) {
            int i, j;
            fold_ij(f, 2 * m, i, j);
            Lv[gpidx(2 * m, i, j)] = UM[gpidx(D0, 2 * kl + i, 2 * kl + j)];
        }
        __syncthreads();
        // forward: pivots of every level, children of every level but the last
        for (int l = 0; l < m; ++l) {
            const int d = 2 * (m - l), dc = d - 2, np = 1 << l, st = gsym(d), stc = gsym(dc);
            const dd *Lp = Lv + lvl_off(l);
            for (int c = t; c < np; c += kTreeThreads) {
                const dd *P = Lp + c * st;
                const dd p00 = P[gpidx(d, 0, 0)], p01 = P[gpidx(d, 0, 1)], p11 = P[gpidx(d, 1, 1)];
                const dd det = dd_dot2(p00, p11, -p01, p01);
                const dd rs = dd_rsqrt(det), inv = rs * rs;
                const int node = np - 1 + c;
                nQ[3 * node] = p11 * inv;
                nQ[3 * node + 1] = -p01 * inv;
                nQ[3 * node + 2] = p00 * inv;
                nrs[node] = rs;
                if (!(det.hi > 0.0)) atomicOr(&s_bad, 1);
            }
            __syncthreads();
            if (l == m - 1) break;
            for (int f = t; f < np * dc; f += kTreeThreads) {
                const int cp = f / dc, i = f - cp * dc, node = np - 1 + cp;
                const dd *P = Lp + cp * st;
                const dd b0 = P[gpidx(d, 0, i + 2)], b1 = P[gpidx(d, 1, i + 2)];
                const dd q00 = nQ[3 * node], q01 = nQ[3 * node + 1], q11 = nQ[3 * node + 2];
                Yb[2 * f] = dd_dot2(q00, b0, q01, b1);
                Yb[2 * f + 1] = dd_dot2(q01, b0, q11, b1);
            }
            __syncthreads();
            dd *Lc = Lv + lvl_off(l + 1);
            for (int f = t; f < np * stc; f += kTreeThreads) {
                const int cp = f / stc, e = f - cp * stc;
                int i, j;
                fold_ij(e, dc, i, j);
                const dd *P = Lp + cp * st;
                const dd *W = Yb + 2 * (cp * dc + i);
                const dd v = P[gpidx(d, i + 2, j + 2)];
                Lc[(2 * cp) * stc + gpidx(dc, i, j)] = v;
                Lc[(2 * cp + 1) * stc + gpidx(dc, i, j)] =
                    dd_fms2(v, W[0], P[gpidx(d, 0, j + 2)], W[1], P[gpidx(d, 1, j + 2)]);
            }
            __syncthreads();
        }
        // subtree sums, leaves up
        for (int l = m - 1; l >= 0; --l) {
            const int np = 1 << l;
            for (int c = t; c < np; c += kTreeThreads) {
                const int node = np - 1 + c;
                if (l == m - 1) {
                    nS[node] = nrs[node] - dd(1.0);
                } else {
                    const int ch = 2 * np - 1 + 2 * c;  // exclude child; ch + 1 includes
                    nS[node] = nrs[node] * nS[ch + 1] - nS[ch];
                }
            }
            __syncthreads();
        }
        if (t == 0) {
            dd V = tau * nS[0];
            if ((q - k) & 1) V = -V;
            s_V = V;
            s_T += V;
        }
        __syncthreads();
        const dd V = s_V;
        // reverse through the subtree: the last level's pivot blocks, then upwards
        dd *Ach = base + ((m - 1) & 1 ? kOffAdjB : kOffAdjA);
        for (int c = t; c < (1 << (m - 1)); c += kTreeThreads) {
            const int node = (1 << (m - 1)) - 1 + c;
            const dd h = nrs[node] * dd(-0.5);
            Ach[3 * c] = h * nQ[3 * node];
            Ach[3 * c + 1] = h * nQ[3 * node + 1];
            Ach[3 * c + 2] = h * nQ[3 * node + 2];
        }
        __syncthreads();
        for (int l = m - 2; l >= 0; --l) {
            const int d = 2 * (m - l), dc = d - 2, np = 1 << l, st = gsym(d), stc = gsym(dc);
            const dd *Lp = Lv + lvl_off(l);
            const dd *Ac = base + ((l + 1) & 1 ? kOffAdjB : kOffAdjA);
            dd *Ap = base + (l & 1 ? kOffAdjB : kOffAdjA);
            // Y = P^{-1} B Gamma(inc), one column j per job
            for (int f = t; f < np * dc; f += kTreeThreads) {
                const int cp = f / dc, j = f - cp * dc, node = np - 1 + cp;
                const dd *P = Lp + cp * st;
                const dd *Gi = Ac + (2 * cp + 1) * stc;
                dd z0 = dd(0.0), z1 = dd(0.0);
                for (int i = 0; i < dc; ++i) {
                    const dd g = Gi[gpany(dc, i, j)];
                    z0 = z0 + P[gpidx(d, 0, i + 2)] * g;
                    z1 = z1 + P[gpidx(d, 1, i + 2)] * g;
                }
                const dd q00 = nQ[3 * node], q01 = nQ[3 * node + 1], q11 = nQ[3 * node + 2];
                Yb[2 * f] = dd_dot2(q00, z0, q01, z1);
                Yb[2 * f + 1] = dd_dot2(q01, z0, q11, z1);
            }
            __syncthreads();
            for (int f = t; f < np * st; f += kTreeThreads) {
                const int cp = f / st, e = f - cp * st, node = np - 1 + cp;
                int i, j;
                fold_ij(e, d, i, j);
                const dd rs = nrs[node];
                dd g;
                if (i >= 2) {
                    g = rs * Ac[(2 * cp + 1) * stc + gpidx(dc, i - 2, j - 2)] - Ac[(2 * cp) * stc + gpidx(dc, i - 2, j - 2)];
                } else if (j >= 2) {
                    g = -(rs * Yb[2 * (cp * dc + j - 2) + i]);
                } else {
                    // (Y B^T P^{-1})(i, j) - S(inc) P^{-1}(i, j) / 2, times rs
                    const dd *P = Lp + cp * st;
                    dd yb0 = dd(0.0), yb1 = dd(0.0);
                    for (int c = 0; c < dc; ++c) {
                        const dd y = Yb[2 * (cp * dc + c) + i];
                        yb0 = yb0 + y * P[gpidx(d, 0, c + 2)];
                        yb1 = yb1 + y * P[gpidx(d, 1, c + 2)];
                    }
                    const dd qj0 = nQ[3 * node + (j == 0 ? 0 : 1)], qj1 = nQ[3 * node + (j == 0 ? 1 : 2)];
                    const dd qij = nQ[3 * node + i + j];
                    g = rs * (dd_dot2(yb0, qj0, yb1, qj1) - nS[2 * np - 1 + 2 * cp + 1] * qij * dd(0.5));
                }
                Ap[cp * st + gpidx(d, i, j)] = g;
            }
            __syncthreads();
        }
        // the unit's adjoint: the root's, scaled, then back through its low pivots, then
        // into Gam at the unit's rows
        {
            const dd fac = (((q - k) & 1) ? -tau : tau);
            const dd *Ar = base + kOffAdjA;  // level 0
            for (int f = t; f < gsym(2 * m); f += kTreeThreads) {
                int i, j;
                fold_ij(f, 2 * m, i, j);
                Gf[gpidx(D0, 2 * kl + i, 2 * kl + j)] = fac * Ar[gpidx(2 * m, i, j)];
            }
        }
        __syncthreads();
        reverse_pivots(UM, Gf, D0, kl, preQ, V, Yb);
        for (int f = t; f < gsym(D0); f += kTreeThreads) {
            int i, j;
            fold_ij(f, D0, i, j);
            dd &g = Gam[gpidx(Dr, umrow[i], umrow[j])];
            g = g + Gf[gpidx(D0, i, j)];
        }
        __syncthreads();
    }
    // the chunk: Gam as the adjoint of SM's trailing block, back through the high pivots
    // with the chunk's sum as their V
    for (int f = t; f < gsym(Dr); f += kTreeThreads) {
        int i, j;
        fold_ij(f, Dr, i, j);
        Gs[gpidx(Ds, 2 * kh + i, 2 * kh + j)] = Gam[gpidx(Dr, i, j)];
    }
    __syncthreads();
    reverse_pivots(SM, Gs, Ds, kh, hiQ, s_T, Yb);
    // dense partial (row stride 2n): zero, then the chunk's rows
    for (int f = t; f < Dn * Dn; f += kTreeThreads) {
        part_hi[ch * pst + f] = 0.0;
        part_lo[ch * pst + f] = 0.0;
    }
    __syncthreads();
    for (int f = t; f < gsym(Ds); f += kTreeThreads) {
        int i, j;
        fold_ij(f, Ds, i, j);
        const dd g = Gs[gpidx(Ds, i, j)];
        const int ri = smrow[i], rj = smrow[j];
        part_hi[ch * pst + (size_t)ri * Dn + rj] = g.hi;
        part_lo[ch * pst + (size_t)ri * Dn + rj] = g.lo;
        part_hi[ch * pst + (size_t)rj * Dn + ri] = g.hi;
        part_lo[ch * pst + (size_t)rj * Dn + ri] = g.lo;
    }
    if (t == 0) {
        part_T[2 * ch] = s_T.hi;
        part_T[2 * ch + 1] = s_T.lo;
        if (s_bad) atomicOr(flags + p, 1);
    }
}

// per pattern: sum the chunk partials in order, F_p = (w_p / T_p) Gbar_p, log P_p
__global__ void grad_finalize_kernel(int M, const uint64_t *__restrict__ pats, int n_pat,
                                     const long long *__restrict__ chunk_off, size_t pst,
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
            s += dd(part_hi[(size_t)c * pst + f], part_lo[(size_t)c * pst + f]);
        F[(size_t)p * kGD * kGD + f] = (s.hi + s.lo) * s_scale;
    }
}

// H[i][j] = sum_p F_p at the rows of S_p (patterns in order: deterministic); sumw
__global__ void grad_scatter_kernel(int M, const uint64_t *__restrict__ pats, int n_pat,
                                    const double *__restrict__ F, size_t fst, const double *__restrict__ w,
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
        h += F[(size_t)p * fst + (2 * rank(mi) + ai) * D + (2 * rank(mj) + aj)];
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
    int layer = 0, base = 0;
    for (;;) {
        int cnt = (M - 1 - (layer & 1) + 1) / 2;  // m = parity, parity+2, ... < M - 1
        if (c < base + cnt) return (layer & 1) + 2 * (c - base);
        base += cnt;
        ++layer;
    }
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

// one partial per pattern
size_t al(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

int grad_sigmaQ(gbs_ctx *ctx, int M, const double *O, const double *logdet, const uint64_t *pats,
                int n_pat, const double *w, double *dsq, double *logP, int32_t *status) {
    // every pattern must be valid and have at most kGradMaxN clicks: checked on the host
    // from a copy of the pattern words (one small readback), which also sizes the chunks
    size_t pb = (size_t)n_pat * 16;
    uint64_t *hp = (uint64_t *)malloc(pb + 16);
    if (!hp) return gbs_fail(ctx, GBS_E_NOMEM, "gbs_grad: host buffer");
    GBS_CUDA(ctx, cudaMemcpyAsync(hp, pats, pb, cudaMemcpyDeviceToHost, ctx->stream));
    GBS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    long long total_units = 0;
    int n_max = 0;
    for (int p = 0; p < n_pat; ++p) {
        uint64_t lo = hp[2 * p], hi = hp[2 * p + 1];
        int n = __builtin_popcountll(lo) + __builtin_popcountll(hi);
        bool out_of_range = (M < 64 && (lo >> M)) || (M <= 64 && hi) || (M > 64 && M < 128 && (hi >> (M - 64)));
        if (n > kGradMaxN || out_of_range) {
            free(hp);
            return gbs_fail(ctx, GBS_E_INVALID, "gbs_grad: pattern %d has %d clicks (at most %d) or a detector >= M",
                            p, n, kGradMaxN);
        }
        total_units += 1ll << (n > kTM ? n - kTM : 0);
        n_max = n > n_max ? n : n_max;
    }
    // chunks: aligned runs of `per` = 2^b consecutive units of one pattern (all of them if it
    // has fewer), b sized for about 32 chunks per SM over the whole batch and at most
    // kChunkBits: the largest patterns no longer set the time of the launch alone, and the
    // more of the prefix modes are fixed within a chunk, the more pivots its units share
    // (82 ms against 109 ms with 8 chunks per SM on the 32-mode workload)
    const long long target = 32ll * ctx->num_sms;
    long long per = 1;
    while (per < (1ll << kChunkBits) && per * target < total_units) per *= 2;
    long long chunks = 0;
    for (int p = 0; p < n_pat; ++p) {
        const int n = __builtin_popcountll(hp[2 * p]) + __builtin_popcountll(hp[2 * p + 1]);
        const long long units = 1ll << (n > kTM ? n - kTM : 0);
        chunks += (units + per - 1) / per;
    }
    const size_t tb = sizeof(long long) * ((size_t)n_pat + 1) + sizeof(long long) * 2 * (size_t)chunks +
                      sizeof(int) * (size_t)chunks;
    char *ht = (char *)malloc(tb);
    if (!ht) {
        free(hp);
        return gbs_fail(ctx, GBS_E_NOMEM, "gbs_grad: host buffer");
    }
    long long *h_off = (long long *)ht, *h_u = h_off + (n_pat + 1);
    int *h_p = (int *)(h_u + 2 * chunks);
    long long c = 0;
    for (int p = 0; p < n_pat; ++p) {
        const int n = __builtin_popcountll(hp[2 * p]) + __builtin_popcountll(hp[2 * p + 1]);
        const long long units = 1ll << (n > kTM ? n - kTM : 0);
        h_off[p] = c;
        for (long long u0 = 0; u0 < units; u0 += per, ++c) {
            h_p[c] = p;
            h_u[2 * c] = u0;
            h_u[2 * c + 1] = u0 + per < units ? u0 + per : units;
        }
    }
    h_off[n_pat] = c;
    free(hp);
    const int N = 2 * M;
    const size_t pst = (size_t)(2 * n_max) * (2 * n_max);  // one chunk's dense partial (row stride 2n)
    size_t o_off = 0, o_cu = al(o_off + 8 * ((size_t)n_pat + 1)), o_cp = al(o_cu + 16 * (size_t)chunks),
           o_flags = al(o_cp + 4 * (size_t)chunks), o_phi = al(o_flags + 4 * (size_t)n_pat),
           o_plo = al(o_phi + 8 * (size_t)chunks * pst), o_pT = al(o_plo + 8 * (size_t)chunks * pst),
           o_F = al(o_pT + 16 * (size_t)chunks), o_H = al(o_F + 8 * (size_t)n_pat * kGD * kGD),
           o_T1 = al(o_H + 8 * (size_t)N * N), o_T2 = al(o_T1 + 8 * (size_t)N * N), o_sw = al(o_T2 + 8 * (size_t)N * N),
           total = o_sw + 64;
    int st = gbs_ws_ensure(ctx, total);
    if (st) {
        free(ht);
        return st;
    }
    char *b = (char *)ctx->ws;
    long long *chunk_off = (long long *)(b + o_off), *chunk_u = (long long *)(b + o_cu);
    int *chunk_p = (int *)(b + o_cp);
    int *flags = (int *)(b + o_flags);
    double *phi_ = (double *)(b + o_phi), *plo = (double *)(b + o_plo), *pT = (double *)(b + o_pT);
    double *F = (double *)(b + o_F), *H = (double *)(b + o_H), *T1 = (double *)(b + o_T1),
           *T2 = (double *)(b + o_T2), *sw = (double *)(b + o_sw);
    // the chunk table (copied before the host buffer is released)
    cudaError_t ce = cudaMemcpyAsync(chunk_off, h_off, sizeof(long long) * ((size_t)n_pat + 1),
                                     cudaMemcpyHostToDevice, ctx->stream);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(chunk_u, h_u, sizeof(long long) * 2 * (size_t)chunks, cudaMemcpyHostToDevice, ctx->stream);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(chunk_p, h_p, sizeof(int) * (size_t)chunks, cudaMemcpyHostToDevice, ctx->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
    free(ht);
    GBS_CUDA(ctx, ce);
    GBS_CUDA(ctx, cudaMemsetAsync(flags, 0, sizeof(int) * (size_t)n_pat, ctx->stream));
    const size_t smem = sizeof(dd) * (size_t)kTreeSmem;
    GBS_CUDA(ctx, cudaFuncSetAttribute(grad_tree_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    st = gbs_timing_begin(ctx);
    if (st) return st;
    grad_tree_kernel<<<(unsigned)chunks, kTreeThreads, smem, ctx->stream>>>(M, O, pats, n_pat, chunk_p, chunk_u,
                                                                           pst, phi_, plo, pT, flags);
    GBS_CUDA(ctx, cudaGetLastError());
    st = gbs_timing_end(ctx);
    if (st) return st;
    grad_finalize_kernel<<<n_pat, 256, 0, ctx->stream>>>(M, pats, n_pat, chunk_off, pst, phi_, plo, pT, w, logdet, F,
                                                         logP, status, flags);
    GBS_CUDA(ctx, cudaGetLastError());
    return grad_chain_sigma(ctx, M, O, pats, n_pat, F, (size_t)kGD * kGD, w, H, T1, T2, sw, dsq);
}

int grad_chain_sigma(gbs_ctx *ctx, int M, const double *O, const uint64_t *pats, int n_pat, const double *F,
                     size_t fst, const double *w, double *H, double *T1, double *T2, double *sw, double *dsq) {
    const int N = 2 * M;
    dim3 blk(16, 16), grd((N + 15) / 16, (N + 15) / 16);
    grad_scatter_kernel<<<grd, blk, 0, ctx->stream>>>(M, pats, n_pat, F, fst, w, H, sw);
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
