// Exact signed subset sweep (Methods, "Probability of any sample", Eq. (p(n))):
//
//   T(S) = sum_{Z subset S} (-1)^{|S|-|Z|} det(A_Z)^{-1/2},   A = I - O = sigma_Q^{-1},
//   log P(S) = -1/2 log det sigma_Q + log T(S).
//
// The paper evaluates one determinant per subset ("2^n determinants").  Here the
// subsets are the leaves of a binary include/exclude tree over the n modes of S
// and the determinants share their factorisations: at a tree node the Schur
// complement C of the modes already included is kept; excluding the next mode
// drops its two rows (a view, no arithmetic), including it multiplies the
// determinant by det(P) of its 2x2 pivot block and applies the rank-2 update
// C' = C_rest - B P^{-1} B^T.  That is ~44 flops per subset (~50 as executed) instead of
// (2|Z|)^3/3 for a fresh Cholesky.
//
// Work decomposition (one persistent launch over every pattern):
//   unit     = (pattern, include/exclude choice of the first q - s modes): a CTA gathers
//              A on the unit's modes and eliminates the included prefix modes;
//   sub-unit = a choice for the next s modes, the leaves of an s-level tree walked depth
//              first over the unit's trailing block (an include's Schur complement
//              stored per depth, an exclude a view of it); each sub-unit's matrix is
//              expanded L levels breadth-first in shared memory (2^L nodes), then every
//              thread runs the last B levels of its node as straight-line code with the
//              Schur complements in registers.
// Signed terms are accumulated per thread with the error-free TwoSum (float-float
// in the FP32 path, double-double in the FP64 path), reduced across the CTA in
// double with TwoSum, stored per unit, and summed per pattern in unit order.
#include <stdlib.h>

#include <type_traits>

#include "dd.cuh"
#include "fx.cuh"
#include "fx6.cuh"
#include "gbs_internal.cuh"
#include "zc.cuh"

namespace {

constexpr int kL = 7;                  // breadth-first levels per sub-unit
constexpr int kThreads = 1 << kL;      // one thread per node after the expansion
constexpr int kS = 3;                  // prefix levels a CTA loops over inside one unit
constexpr int kMaxN = 40;              // clicks per pattern on the exact path
constexpr int kPlanThreads = 1024;
// whole-device sweeps (all 2^M subsets of one device): 2^36 subsets is about a minute per
// double-double sweep and a 5 GB table of unit bins; beyond that the table alone outgrows
// a sensible workspace (88 GB at M = 40)
constexpr int kMaxDevice = 36;

__host__ __device__ constexpr int sym(int d) { return d * (d + 1) / 2; }
// packed upper-triangle index of (i, j), i <= j, in a d x d symmetric matrix
__host__ __device__ constexpr int pidx(int d, int i, int j) { return i * d - (i * (i - 1)) / 2 + (j - i); }
// odd node stride: per-thread node reads hit distinct banks
__host__ __device__ constexpr int nstride(int d) { return sym(d) | 1; }

// Per precision: B register-resident levels per thread; Tau, the type of the
// products of pivot factors above the thread level; u, the unit roundoff.
template <typename T> struct Prec;
template <> struct Prec<float> {
    static constexpr int B = 6, idx = GBS_FP32_SPLIT;
    using Tau = double;
    using Abs = float;
    using Node = float;
    static constexpr bool fixed = false;
    static constexpr int wrow = 2;  // entries per row of W
    static constexpr double u = 5.9604644775390625e-08, u_sum = 1.1102230246251565e-16;
};
template <> struct Prec<double> {
    static constexpr int B = 4, idx = GBS_FP64;
    using Tau = double;
    using Abs = double;
    using Node = double;
    static constexpr bool fixed = false;
    static constexpr int wrow = 2;
    static constexpr double u = 1.1102230246251565e-16, u_sum = 1.1102230246251565e-16;
};
template <> struct Prec<dd> {
    static constexpr int B = 3, idx = GBS_DD;
    using Tau = dd;
    using Abs = double;
    using Node = dd;
    static constexpr bool fixed = false;
    static constexpr int wrow = 2;
    static constexpr double u = 1.2325951644078309e-32, u_sum = 1.2325951644078309e-32;
};
// Q16.112 fixed point: truncated products (2^-112) and the pivot rsqrt (residual
// 1 - x y^2 within 2^-108) give each factor a relative error far below 2^-100 while its
// pivot determinant stays >= 2^-8; prefactors and sums in double-double.
template <> struct Prec<fx> {
    static constexpr int B = 2, idx = GBS_FX;
    using Tau = dd;
    using Abs = float;
    using Node = fxe;  // prefactors m 2^e
    static constexpr bool fixed = true;
    static constexpr int wrow = 3;  // offset rows (u'0, u'1, t) of U = B R^{-T}
    using Piv = fx_piv;
    static constexpr double u = 7.888609052210118e-31, u_sum = 1.2325951644078309e-32;
};
// Q16.176 fixed point (fx6.cuh): the same sweep 64 bits wider, per-term relative error far
// below 2^-164; prefactors, sub-unit and unit sums as m 2^e with 192-bit mantissas (fxe6)
// and the unit partials summed exactly per pattern, for sums that cancel beyond ~1e20.
template <> struct Prec<fx6> {
    static constexpr int B = 2, idx = GBS_FX192;
    using Tau = fxe6;
    using Abs = float;
    using Node = fxe6;
    static constexpr bool fixed = true;
    static constexpr int wrow = 3;
    using Piv = fx6_piv;
    static constexpr double u = 4.2351647362715017e-50, u_sum = 6.617444900424222e-52;  // 2^-164, 2^-170
};
// doubles per unit partial: (hi, lo, sum |terms|), or the 192-bit fxe6 sum (mantissa in three
// words, exponent) and sum |terms| for fx6
template <typename T> constexpr int partial_words() { return std::is_same<T, fx6>::value ? 5 : 3; }

// Complex FP64 (the sector-resolved binned sweep at a complex generating variable t):
// the matrices I - t O_Z are accretive for |t| <= 1, so the unpivoted recursion is safe and
// the product of the principal det^{-1/2} of the pivot blocks is the principal branch of
// the whole (it is continuous in t and real positive at t = 0).
template <> struct Prec<zc> {
    static constexpr int B = 3;
    using Tau = zc;
    using Abs = double;
    using Node = zc;
    static constexpr bool fixed = false;
    static constexpr int wrow = 2;
};

template <> struct Prec<zf> {
    static constexpr int B = 3;
    using Tau = zf;
    using Abs = double;
    using Node = zf;
    static constexpr bool fixed = false;
    static constexpr int wrow = 2;
};

template <typename T> __device__ __forceinline__ T rsq(T x);
template <> __device__ __forceinline__ zc rsq<zc>(zc x) { return zc_rsqrt(x); }
template <> __device__ __forceinline__ zf rsq<zf>(zf x) { return zf_rsqrt(x); }
template <> __device__ __forceinline__ float rsq<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsq<double>(double x) { return rsqrt(x); }
template <> __device__ __forceinline__ dd rsq<dd>(dd x) { return dd_rsqrt(x); }
template <> __device__ __forceinline__ fx rsq<fx>(fx x) { return fx_rsqrt(x); }
template <> __device__ __forceinline__ fx6 rsq<fx6>(fx6 x) { return fx6_rsqrt(x); }

// 1/sqrt(det) as a prefix factor, in the Tau type of the precision, given rs = rsq(det)
// (FP32 prefactors are taken in FP64)
__device__ __forceinline__ double tau_of(float det, float) { return rsqrt((double)det); }
__device__ __forceinline__ double tau_of(double, double rs) { return rs; }
__device__ __forceinline__ dd tau_of(dd, dd rs) { return rs; }
__device__ __forceinline__ dd tau_of(fx, fx rs) { return fx_to_dd(rs); }
__device__ __forceinline__ fxe6 tau_of(fx6, fx6 rs) { return fxe6_from(rs); }
__device__ __forceinline__ zc tau_of(zc, zc rs) { return rs; }
__device__ __forceinline__ zf tau_of(zf, zf rs) { return rs; }

// constants and conversions of the working type
template <typename T> __device__ __forceinline__ T konst(double v) { return T(v); }
template <> __device__ __forceinline__ fx konst<fx>(double v) { return fx_from_double(v); }
template <> __device__ __forceinline__ fx6 konst<fx6>(double v) { return fx6_from_double(v); }
__device__ __forceinline__ float to_node(float x) { return x; }
__device__ __forceinline__ double to_node(double x) { return x; }
__device__ __forceinline__ dd to_node(dd x) { return x; }
__device__ __forceinline__ zc to_node(zc x) { return x; }
__device__ __forceinline__ zf to_node(zf x) { return x; }
// a child's prefactor: the parent's times det^{-1/2} of the parent's pivot
template <typename N, typename T> __device__ __forceinline__ N node_times(const N &p, const T &rs) { return p * to_node(rs); }
template <> __device__ __forceinline__ fxe node_times<fxe, fx>(const fxe &p, const fx &rs) { return fxe_mul(p, rs); }
template <typename N> __device__ __forceinline__ N node_one() { return N(1.0); }
template <> __device__ __forceinline__ fxe node_one<fxe>() { return fxe_one(); }
template <> __device__ __forceinline__ fxe6 node_one<fxe6>() { return fxe6(1.0); }
template <> __device__ __forceinline__ fxe6 node_times<fxe6, fx6>(const fxe6 &p, const fx6 &rs) { return fxe_mul(p, rs); }
// product of two non-negative factors
template <typename T> __device__ __forceinline__ T mul_pos(T a, T b) { return a * b; }
template <> __device__ __forceinline__ fx mul_pos<fx>(fx a, fx b) { return fx_mul_uu(a, b); }
template <> __device__ __forceinline__ fx6 mul_pos<fx6>(fx6 a, fx6 b) { return fx_mul_uu(a, b); }
// pivot check: 0 fine, 1 not positive (or NaN), 2 outside the fixed-point range
template <typename T> __device__ __forceinline__ int pivot_bad(T det) { return det > T(0) ? 0 : 1; }
template <> __device__ __forceinline__ int pivot_bad<fx>(fx det) { return fx_pivot_bad(det); }
template <> __device__ __forceinline__ int pivot_bad<fx6>(fx6 det) { return fx_pivot_bad(det); }
// complex pivots: their determinants may have any argument in (-pi, pi); only zero or NaN is bad
template <> __device__ __forceinline__ int pivot_bad<zc>(zc det) {
    return fabs(det.re) + fabs(det.im) > 0.0 ? 0 : 1;
}
template <> __device__ __forceinline__ int pivot_bad<zf>(zf det) {
    return fabsf(det.re.hi) + fabsf(det.im.hi) > 0.0f ? 0 : 1;
}

// the Schur-update kernels: a0 b0 + a1 b1, c - a0 b0 - a1 b1, det of a 2x2 block
template <typename T> __device__ __forceinline__ T dot2(T a0, T b0, T a1, T b1) { return a0 * b0 + a1 * b1; }
template <> __device__ __forceinline__ dd dot2<dd>(dd a0, dd b0, dd a1, dd b1) { return dd_dot2(a0, b0, a1, b1); }
template <typename T> __device__ __forceinline__ T fms2(T c, T a0, T b0, T a1, T b1) { return c - a0 * b0 - a1 * b1; }
template <> __device__ __forceinline__ dd fms2<dd>(dd c, dd a0, dd b0, dd a1, dd b1) { return dd_fms2(c, a0, b0, a1, b1); }
template <typename T> __device__ __forceinline__ T det2(T p00, T p01, T p11) { return dot2(p00, p11, -p01, p01); }
template <> __device__ __forceinline__ fx det2<fx>(fx p00, fx p01, fx p11) { return fx_det2(p00, p01, p11); }
template <> __device__ __forceinline__ fx6 det2<fx6>(fx6 p00, fx6 p01, fx6 p11) { return fx_det2(p00, p01, p11); }

// an entry of A = I - O from its FP64 data (exact in double-double)
template <typename T> __device__ __forceinline__ T a_entry(double delta, double o) { return (T)(delta - o); }
template <> __device__ __forceinline__ dd a_entry<dd>(double delta, double o) { return dd_two_sum(delta, -o); }
template <> __device__ __forceinline__ fx a_entry<fx>(double delta, double o) {
    return fx_from_double(delta) - fx_from_double(o);
}
template <> __device__ __forceinline__ fx6 a_entry<fx6>(double delta, double o) {
    return fx6_from_double(delta) - fx6_from_double(o);
}

// the same with the generating variable t of the complex binned sweep: I - t O
template <typename T> __device__ __forceinline__ T a_entry_t(double delta, double o, double, double) {
    return a_entry<T>(delta, o);
}
template <> __device__ __forceinline__ zc a_entry_t<zc>(double delta, double o, double t_re, double t_im) {
    return zc(delta - t_re * o, -t_im * o);
}
template <> __device__ __forceinline__ zf a_entry_t<zf>(double delta, double o, double t_re, double t_im) {
    return zf(ff(delta - t_re * o), ff(-t_im * o));
}

__device__ __forceinline__ double to_hi(float x) { return x; }
__device__ __forceinline__ double to_hi(double x) { return x; }
// leading part of a (positive) term, in the type its magnitude is summed in
__device__ __forceinline__ float abs_part(float x) { return x; }
__device__ __forceinline__ double abs_part(double x) { return x; }
__device__ __forceinline__ double abs_part(dd x) { return x.hi; }
__device__ __forceinline__ float abs_part(fx x) { return (float)(int32_t)x.w[3] * (1.0f / 65536.0f); }
__device__ __forceinline__ float abs_part(fx6 x) { return (float)(int32_t)x.w[5] * (1.0f / 65536.0f); }
__device__ __forceinline__ bool is_nan(float x) { return x != x; }
__device__ __forceinline__ bool is_nan(double x) { return x != x; }
__device__ __forceinline__ bool is_nan(dd x) { return x.hi != x.hi; }
__device__ __forceinline__ bool is_nan(zc x) { return zc_nan(x); }
__device__ __forceinline__ bool is_nan(zf x) { return zf_nan(x); }
// a thread's subtree sum as (hi, lo) doubles
__device__ __forceinline__ void sum_parts(float h, float l, double &oh, double &ol) { oh = h; ol = l; }
__device__ __forceinline__ void sum_parts(double h, double l, double &oh, double &ol) { oh = h; ol = l; }
__device__ __forceinline__ void sum_parts(dd h, dd l, double &oh, double &ol) { oh = h.hi; ol = h.lo + l.hi; }

// ---- prefactor arrays --------------------------------------------------------------
// The node prefactors are stored packed: a fixed-point m 2^e as its mantissa words and
// exponent (20 or 28 bytes), every other type as itself.
template <typename N> struct NodeIO {
    static constexpr int bytes = sizeof(N), align = alignof(N);
    static __device__ __forceinline__ N ld(const unsigned char *b, int i) { return ((const N *)b)[i]; }
    static __device__ __forceinline__ void st(unsigned char *b, int i, const N &v) { ((N *)b)[i] = v; }
};
template <> struct NodeIO<fxe> {
    static constexpr int bytes = 20, align = 4;
    static __device__ __forceinline__ fxe ld(const unsigned char *b, int i) {
        const uint32_t *q = (const uint32_t *)(b + bytes * i);
        fxe r;
#pragma unroll
        for (int k = 0; k < 4; ++k) r.m.w[k] = q[k];
        r.e = (int)q[4];
        return r;
    }
    static __device__ __forceinline__ void st(unsigned char *b, int i, const fxe &v) {
        uint32_t *q = (uint32_t *)(b + bytes * i);
#pragma unroll
        for (int k = 0; k < 4; ++k) q[k] = v.m.w[k];
        q[4] = (uint32_t)v.e;
    }
};
template <> struct NodeIO<fxe6> {
    static constexpr int bytes = 28, align = 4;
    static __device__ __forceinline__ fxe6 ld(const unsigned char *b, int i) {
        const uint32_t *q = (const uint32_t *)(b + bytes * i);
        fxe6 r;
#pragma unroll
        for (int k = 0; k < 6; ++k) r.m.w[k] = q[k];
        r.e = (int)q[6];
        return r;
    }
    static __device__ __forceinline__ void st(unsigned char *b, int i, const fxe6 &v) {
        uint32_t *q = (uint32_t *)(b + bytes * i);
#pragma unroll
        for (int k = 0; k < 6; ++k) q[k] = v.m.w[k];
        q[6] = (uint32_t)v.e;
    }
};

// ---- shared-memory layout ----------------------------------------------------
// X and Y alternate as source and destination of the breadth-first levels; the
// unit's prefix-elimination matrix (up to 2 kMaxN rows) spans X, Y, Ub and W before
// the levels start.  Ub holds the unit's trailing block, Sl the sub-unit tree's stored
// matrices, W the rows W = B P^{-1} of the level being eliminated; a level's pivot
// quantities sit at the start of its destination buffer (read before the children are
// written).  The prefactor arrays hold the W rows of a prefix pivot.
template <typename T> struct Layout {
    static constexpr int B = Prec<T>::B;
    static constexpr int R = kL + B;  // modes of a unit's level-0 matrix
    static constexpr int level_size(int l) { return (1 << l) * nstride(2 * (R - l)); }
    static constexpr int max_even() {
        int m = 0;
        for (int l = 0; l <= kL; l += 2) m = level_size(l) > m ? level_size(l) : m;
        return m;
    }
    static constexpr int max_odd() {
        int m = 0;
        for (int l = 1; l <= kL; l += 2) m = level_size(l) > m ? level_size(l) : m;
        return m;
    }
    static constexpr int w_entries() {
        int m = 0;
        for (int l = 0; l < kL; ++l) {
            const int v = (1 << l) * Prec<T>::wrow * (2 * (R - l - 1));
            m = v > m ? v : m;
        }
        return m;
    }
    static constexpr int dec_entries() {
        int s = 0;
        for (int m = 1; m <= R; ++m) s += sym(2 * m);
        return s;
    }
    // byte offsets
    using Node = typename Prec<T>::Node;
    static constexpr size_t off_X = 0;
    static constexpr size_t off_Y = off_X + sizeof(T) * max_even();
    static constexpr int ublk() { return sym(2 * (kS + R)); }
    static constexpr size_t off_U = off_Y + sizeof(T) * max_odd();
    // the sub-unit tree's stored matrices: after an include at depth d < kS - 1, the
    // 2 (kS + R - d - 1) rows of the modes below it
    static constexpr int slot_off(int d) {
        int o = 0;
        for (int e = 1; e < d; ++e) o += sym(2 * (kS + R - e));
        return o;
    }
    static constexpr size_t off_Sl = off_U + sizeof(T) * ublk();
    static constexpr size_t off_W = off_Sl + sizeof(T) * slot_off(kS);
    // prefactors: even levels hold at most kThreads / 2 nodes, odd levels kThreads
    static constexpr size_t off_tauX = off_W + sizeof(T) * w_entries();
    static constexpr size_t off_tauY = off_tauX + NodeIO<Node>::bytes * (kThreads / 2);
    static constexpr size_t off_red = (off_tauY + NodeIO<Node>::bytes * kThreads + 15) / 16 * 16;  // 3 doubles per warp
    static constexpr size_t off_modes = off_red + sizeof(double) * 3 * (kThreads / 32);
    static constexpr size_t off_pos = off_modes + sizeof(int) * 64;
    static constexpr size_t off_decoff = off_pos + sizeof(int) * 2 * kMaxN;
    static constexpr size_t off_dec = off_decoff + sizeof(int) * (R + 2);
    static constexpr size_t bytes = (off_dec + sizeof(uint16_t) * dec_entries() + 15) / 16 * 16;
    static_assert(sizeof(T) * sym(2 * kMaxN) <= off_tauX, "prefix matrix must fit in X, Y, Ub and W");
    static_assert(sizeof(T) * 2 * (2 * kMaxN - 2) <= off_red - off_tauX, "prefix W rows must fit in the prefactors");
    static_assert(off_Y % alignof(T) == 0 && off_tauX % alignof(T) == 0 && off_tauX % NodeIO<Node>::align == 0 &&
                      off_tauY % NodeIO<Node>::align == 0 && off_red % alignof(double) == 0,
                  "shared-memory regions must be aligned for their types");
};

// ---- error-free accumulation ----------------------------------------------------
__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e) {
    s = a + b;
    double bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}

template <typename T> struct Acc {
    T hi, lo;
    typename Prec<T>::Abs abs;  // sum of |terms|, for kappa only
    int bad;                    // fixed point: pivot checks of the register levels
};

template <typename T> __device__ __forceinline__ void acc_add(Acc<T> &a, T x) {
    T s = a.hi + x;
    T bp = s - a.hi;
    a.lo += (a.hi - (s - bp)) + (x - bp);
    a.hi = s;
}
// double-double sums need no further compensation; fixed-point sums are exact
template <> __device__ __forceinline__ void acc_add<dd>(Acc<dd> &a, dd x) { a.hi += x; }
template <> __device__ __forceinline__ void acc_add<fx>(Acc<fx> &a, fx x) { a.hi += x; }
template <> __device__ __forceinline__ void acc_add<fx6>(Acc<fx6> &a, fx6 x) { a.hi += x; }

// (hi, lo) += sc * (x_hi + x_lo) for one thread's subtree sum
__device__ __forceinline__ void unit_add(double &h, double &l, double sc, double xh, double xl) {
    double s, e;
    two_sum(h, sc * xh, s, e);
    h = s;
    l += e + sc * xl;
}
__device__ __forceinline__ void unit_add(double &h, double &l, dd sc, double xh, double xl) {
    dd c = sc * dd(xh, xl);
    dd u = dd(h, l) + c;
    h = u.hi;
    l = u.lo;
}
__device__ __forceinline__ double tau_abs(double x) { return fabs(x); }
__device__ __forceinline__ double tau_abs(const fxe6 &x) { return fabs(fxe6_to_double(x)); }
__device__ __forceinline__ double tau_abs(dd x) { return fabs(x.hi); }
// (hi, lo) * prefix factor
__device__ __forceinline__ void unit_scale(double &h, double &l, double tp) {
    h *= tp;
    l *= tp;
}
__device__ __forceinline__ void unit_scale(double &h, double &l, dd tp) {
    dd u = dd(h, l) * tp;
    h = u.hi;
    l = u.lo;
}
__device__ __forceinline__ double tau_hi(double x) { return x; }
__device__ __forceinline__ double tau_hi(dd x) { return x.hi; }


// ---- register-resident bottom levels ----------------------------------------------
template <typename T, int MD> struct RegMat {
    T v[sym(2 * MD)];
    __device__ __forceinline__ T operator()(int i, int j) const { return v[pidx(2 * MD, i, j)]; }
};
template <typename T, int MD> struct SmemMat {
    const T *p;
    __device__ __forceinline__ T operator()(int i, int j) const { return p[pidx(2 * MD, i, j)]; }
};

// Subtree of the node whose matrix is A viewed from mode O on (MD - O modes).
// NEG: the node's leaves carry a minus sign relative to the subtree root.
// Levels at depth >= nreal are padding modes (identity block): include only.
// the two leaves of a last-level node: include (+tau rs) and exclude (-tau), signed
// into the subtree sum; or, binned by subset size (cnt = modes included so far in the
// subtree), unsigned into the size bins
template <bool NEG, typename T>
__device__ __forceinline__ void leaf_pair(Acc<T> &acc, T inc, T tau, bool real, int) {
    T comb = real ? inc - tau : inc;
    acc_add(acc, NEG ? -comb : comb);
    acc.abs += real ? abs_part(inc) + abs_part(tau) : abs_part(inc);
}
template <typename T, int NB> struct BinAcc {
    T v[NB];
    int bad;
};
template <bool NEG, typename T, int NB>
__device__ __forceinline__ void leaf_pair(BinAcc<T, NB> &acc, T inc, T tau, bool real, int cnt) {
    acc.v[cnt + 1] += inc;
    if (real) acc.v[cnt] += tau;
}

// ONE: tau is exactly 1 (the subtree root and its exclude-only descendants), so products
// with it are skipped
template <typename T, int MD, int O, bool NEG, bool ONE = true, typename Src, typename AccT>
__device__ __forceinline__ void dfs(const Src &A, T tau, int depth, int nreal, AccT &acc, int cnt) {
    constexpr int m = MD - O;
    constexpr int o = 2 * O;
    const T p00 = A(o, o), p01 = A(o, o + 1), p11 = A(o + 1, o + 1);
    const bool real = depth < nreal;
    if constexpr (m == 1) {
        const T det = det2(p00, p01, p11);
        if constexpr (Prec<T>::fixed) acc.bad |= pivot_bad(det);
        const T rs = rsq<T>(det);
        leaf_pair<NEG>(acc, ONE ? rs : mul_pos(tau, rs), tau, real, cnt);
    } else if constexpr (Prec<T>::fixed) {
        // symmetric form C - U U^T, U = B R^{-T} (offset rows)
        constexpr int d = 2 * (m - 1);
        const typename Prec<T>::Piv v = fx_pivot(p00, p01, p11);
        acc.bad |= fx_chol_bad(p00, v.det);
        T u0[d], u1[d], tt[d];
#pragma unroll
        for (int i = 0; i < d; ++i) fx_urow(v, A(o, o + 2 + i), A(o + 1, o + 2 + i), u0[i], u1[i], tt[i]);
        RegMat<T, m - 1> C;
#pragma unroll
        for (int i = 0; i < d; ++i)
#pragma unroll
            for (int j = i; j < d; ++j)
                C.v[pidx(d, i, j)] = fx_sym_update(A(o + 2 + i, o + 2 + j), u0[i], u1[i], tt[i], u0[j], u1[j], tt[j]);
        dfs<T, m - 1, 0, NEG, false>(C, ONE ? v.rs : fx_mul_uu(tau, v.rs), depth + 1, nreal, acc, cnt + 1);
        if (real) dfs<T, MD, O + 1, !NEG, ONE>(A, tau, depth + 1, nreal, acc, cnt);
    } else {
        constexpr int d = 2 * (m - 1);
        const T det = det2(p00, p01, p11);
        const T rs = rsq<T>(det);
        const T inv = rs * rs;
        const T q00 = p11 * inv, q01 = -p01 * inv, q11 = p00 * inv;
        T b0[d], b1[d], w0[d], w1[d];
#pragma unroll
        for (int i = 0; i < d; ++i) {
            b0[i] = A(o, o + 2 + i);
            b1[i] = A(o + 1, o + 2 + i);
            w0[i] = dot2(q00, b0[i], q01, b1[i]);
            w1[i] = dot2(q01, b0[i], q11, b1[i]);
        }
        RegMat<T, m - 1> C;
#pragma unroll
        for (int i = 0; i < d; ++i)
#pragma unroll
            for (int j = i; j < d; ++j)
                C.v[pidx(d, i, j)] = fms2(A(o + 2 + i, o + 2 + j), w0[i], b0[j], w1[i], b1[j]);
        dfs<T, m - 1, 0, NEG, false>(C, ONE ? rs : tau * rs, depth + 1, nreal, acc, cnt + 1);
        if (real) dfs<T, MD, O + 1, !NEG, ONE>(A, tau, depth + 1, nreal, acc, cnt);
    }
}

// ---- plan: order patterns by click count, one unit per prefix choice -----------------
// n_eff = clicks padded to >= B; L_eff breadth-first levels; q prefix levels of
// which the first q - s index units and the last s (s <= split <= kS) are looped over
// in the CTA.  The split sets the work per unit (2^(s + L + B) subsets): the autotuner
// picks it per precision.
template <typename T>
__host__ __device__ inline void unit_shape(int n, int &n_eff, int &L_eff, int &q, int &s, int split) {
    constexpr int B = Prec<T>::B;
    n_eff = n > B ? n : B;
    L_eff = n_eff - B < kL ? n_eff - B : kL;
    q = n_eff - B - L_eff;
    s = q < split ? q : split;
}

struct Plan {
    unsigned long long *counter;
    long long *total_units;
    int *overflow;      // 1: the batch exceeded the workspace and was not evaluated
    int *perm;          // sorted position -> pattern index
    int *pat_n;         // clicks of each pattern (-1 invalid)
    long long *unit_off;  // n_pat + 1, in sorted order
    int *pflags;        // per sorted position: status bits
    double *partials;   // 3 per unit
    int split;          // prefix levels looped inside a unit (0..kS)
    double t_re, t_im;  // complex binned sweep: the generating variable t of A = I - t O
};

template <typename T>
__global__ void __launch_bounds__(kPlanThreads) plan_kernel(int M, const uint64_t *__restrict__ pats,
                                                           int n_pat, long long cap_units, Plan pl) {
    __shared__ int hist[130];
    __shared__ long long chunk[kPlanThreads];
    const int t = threadIdx.x;
    for (int i = t; i < 130; i += kPlanThreads) hist[i] = 0;
    __syncthreads();
    const uint64_t mlo = M >= 64 ? ~0ull : ((1ull << M) - 1);
    const uint64_t mhi = M > 64 ? (M >= 128 ? ~0ull : ((1ull << (M - 64)) - 1)) : 0ull;
    for (int p = t; p < n_pat; p += kPlanThreads) {
        uint64_t lo = pats[2 * p], hi = pats[2 * p + 1];
        int n = __popcll(lo) + __popcll(hi);
        bool ok = !(lo & ~mlo) && !(hi & ~mhi) && n <= kMaxN;
        int key = ok ? n : -1;
        pl.pat_n[p] = key;
        atomicAdd(&hist[key + 1], 1);
    }
    __syncthreads();
    if (t == 0) {  // bins from the largest n down to the invalid bin
        int run = 0;
        for (int b = 129; b >= 0; --b) {
            int c = hist[b];
            hist[b] = run;
            run += c;
        }
    }
    __syncthreads();
    // stable placement: inside a bin the patterns keep their batch order, so the unit
    // numbering is the same on every call (the batch split of gbs_prob_partial numbers the
    // units of one batch on every rank and relies on it).  Rounds of kPlanThreads patterns:
    // rank inside the warp by __match_any_sync, then per bin an exclusive scan over warps.
    constexpr int kBins = kMaxN + 2;  // keys -1 (invalid) .. kMaxN
    __shared__ int wcnt[kPlanThreads / 32][kBins];
    __shared__ int s_roundtot[kBins];
    for (int base = 0; base < n_pat; base += kPlanThreads) {
        const int p = base + t;
        const int key = p < n_pat ? pl.pat_n[p] + 1 : -1;
        const unsigned grp = __match_any_sync(0xffffffffu, key);
        const int rank_w = __popc(grp & ((1u << (t & 31)) - 1u));
        for (int i = t; i < (kPlanThreads / 32) * kBins; i += kPlanThreads) (&wcnt[0][0])[i] = 0;
        __syncthreads();
        if (key >= 0 && rank_w == 0) wcnt[t >> 5][key] = __popc(grp);
        __syncthreads();
        if (t < kBins) {
            int run = 0;
            for (int w = 0; w < kPlanThreads / 32; ++w) {
                const int c = wcnt[w][t];
                wcnt[w][t] = run;
                run += c;
            }
            s_roundtot[t] = run;
        }
        __syncthreads();
        if (key >= 0) pl.perm[hist[key] + wcnt[t >> 5][key] + rank_w] = p;
        __syncthreads();
        if (t < kBins) hist[t] += s_roundtot[t];
        __syncthreads();
    }
    // unit counts in sorted order, exclusive scan
    const int per = (n_pat + kPlanThreads - 1) / kPlanThreads;
    long long s = 0;
    for (int i = t * per; i < n_pat && i < (t + 1) * per; ++i) {
        int n = pl.pat_n[pl.perm[i]];
        int n_eff, L_eff, q, ss;
        unit_shape<T>(n < 0 ? 0 : n, n_eff, L_eff, q, ss, pl.split);
        s += n < 0 ? 0 : (1ll << (q - ss));
    }
    chunk[t] = s;
    __syncthreads();
    for (int off = 1; off < kPlanThreads; off <<= 1) {
        long long v = t >= off ? chunk[t - off] : 0;
        __syncthreads();
        chunk[t] += v;
        __syncthreads();
    }
    long long run = chunk[t] - s;
    for (int i = t * per; i < n_pat && i < (t + 1) * per; ++i) {
        pl.unit_off[i] = run;
        pl.pflags[i] = 0;
        int n = pl.pat_n[pl.perm[i]];
        int n_eff, L_eff, q, ss;
        unit_shape<T>(n < 0 ? 0 : n, n_eff, L_eff, q, ss, pl.split);
        run += n < 0 ? 0 : (1ll << (q - ss));
    }
    if (t == kPlanThreads - 1) {
        long long total = chunk[t];
        pl.unit_off[n_pat] = total;
        bool over = total > cap_units;
        *pl.total_units = over ? 0 : total;
        *pl.overflow = over ? 1 : 0;
        *pl.counter = 0;
    }
}

// entry f of the upper triangle of a D x D matrix (D even) in (D / 2) (D + 1) folded runs:
// row p and row D - 1 - p share one run of D + 1 entries
__device__ __forceinline__ void fold_ij(int f, int D, int &i, int &j) {
    const int w = D + 1, p = f / w, k = f - p * w;
    if (k < D - p) {
        i = p;
        j = p + k;
    } else {
        i = D - 1 - p;
        j = i + (k - (D - p));
    }
}

// ---- one 2x2 block pivot eliminated by the whole CTA ---------------------------------
// Mx: packed D x D matrix (D even); the pivot block sits on rows c0, c0 + 1.  Rows and
// columns >= c0 + 2 receive C - W B^T, W = B P^{-1} (its rows staged in Wb first).
// Returns 1/sqrt(det P) in the prefix type; a non-positive det sets *flag.
template <typename T>
__device__ __forceinline__ typename Prec<T>::Tau elim_pivot(T *Mx, int D, int c0, T *Wb, int *flag) {
    const int t = threadIdx.x;
    const T p00 = Mx[pidx(D, c0, c0)], p01 = Mx[pidx(D, c0, c0 + 1)], p11 = Mx[pidx(D, c0 + 1, c0 + 1)];
    const T det = det2(p00, p01, p11);
    if (t == 0) {
        const int bad = pivot_bad(det);
        if (bad) atomicOr(flag, bad);
    }
    const int Dt = D - c0 - 2;
    const T rs = rsq<T>(det);
    if (t < Dt) {
        const T inv = rs * rs;
        const T q00 = p11 * inv, q01 = -p01 * inv, q11 = p00 * inv;
        const T b0 = Mx[pidx(D, c0, c0 + 2 + t)], b1 = Mx[pidx(D, c0 + 1, c0 + 2 + t)];
        Wb[2 * t] = dot2(q00, b0, q01, b1);
        Wb[2 * t + 1] = dot2(q01, b0, q11, b1);
    }
    const typename Prec<T>::Tau rt = tau_of(det, rs);
    __syncthreads();
    // the trailing triangle, rows p and Dt - 1 - p folded into one run of Dt + 1 entries
    const int E = (Dt >> 1) * (Dt + 1);
    for (int f = t; f < E; f += kThreads) {
        int i, j;
        fold_ij(f, Dt, i, j);
        T &c = Mx[pidx(D, c0 + 2 + i, c0 + 2 + j)];
        c = fms2(c, Wb[2 * i], Mx[pidx(D, c0, c0 + 2 + j)], Wb[2 * i + 1], Mx[pidx(D, c0 + 1, c0 + 2 + j)]);
    }
    __syncthreads();
    return rt;
}
// The same pivot with the source kept: Dst (packed, D - c0 - 2 rows) receives the
// trailing block's Schur complement, Mx is only read (the same operations in the same
// order as elim_pivot, so the values are those it would leave in place).
template <typename T>
__device__ __forceinline__ typename Prec<T>::Tau elim_into(const T *Mx, int D, int c0, T *Dst, T *Wb, int *flag) {
    const int t = threadIdx.x;
    const T p00 = Mx[pidx(D, c0, c0)], p01 = Mx[pidx(D, c0, c0 + 1)], p11 = Mx[pidx(D, c0 + 1, c0 + 1)];
    const T det = det2(p00, p01, p11);
    if (t == 0) {
        const int bad = pivot_bad(det);
        if (bad) atomicOr(flag, bad);
    }
    const int Dt = D - c0 - 2;
    const T rs = rsq<T>(det);
    if (t < Dt) {
        const T inv = rs * rs;
        const T q00 = p11 * inv, q01 = -p01 * inv, q11 = p00 * inv;
        const T b0 = Mx[pidx(D, c0, c0 + 2 + t)], b1 = Mx[pidx(D, c0 + 1, c0 + 2 + t)];
        Wb[2 * t] = dot2(q00, b0, q01, b1);
        Wb[2 * t + 1] = dot2(q01, b0, q11, b1);
    }
    const typename Prec<T>::Tau rt = tau_of(det, rs);
    __syncthreads();
    const int E = (Dt >> 1) * (Dt + 1);
    for (int f = t; f < E; f += kThreads) {
        int i, j;
        fold_ij(f, Dt, i, j);
        Dst[pidx(Dt, i, j)] = fms2(Mx[pidx(D, c0 + 2 + i, c0 + 2 + j)], Wb[2 * i], Mx[pidx(D, c0, c0 + 2 + j)],
                                   Wb[2 * i + 1], Mx[pidx(D, c0 + 1, c0 + 2 + j)]);
    }
    __syncthreads();
    return rt;
}

// the size bins of the binned mode: double-double sums of real terms, complex sums of
// complex ones
template <typename T> struct BinOf { using type = dd; };
template <> struct BinOf<zc> { using type = zc; };
template <> struct BinOf<zf> { using type = zf; };
__device__ __forceinline__ void store2(double *o, dd v) { o[0] = v.hi; o[1] = v.lo; }
// a thread's bin of the binned mode times its prefactor and the sub-unit factor, in the bin type
template <typename T, typename N, typename Tau> __device__ __forceinline__ typename BinOf<T>::type
scale_bin(const N &tn, const Tau &tsub, T v) {
    return (Tau(tn) * tsub) * v;
}
template <> __device__ __forceinline__ dd scale_bin<fx, fxe, dd>(const fxe &tn, const dd &tsub, fx v) {
    return (fxe_to_dd(tn) * tsub) * fx_to_dd(v);
}
__device__ __forceinline__ bool node_nan(const fxe &) { return false; }
template <typename N> __device__ __forceinline__ bool node_nan(const N &x) { return is_nan(x); }
__device__ __forceinline__ void store2(double *o, zc v) { o[0] = v.re; o[1] = v.im; }
__device__ __forceinline__ void store2(double *o, zf v) { o[0] = ff_to_double(v.re); o[1] = ff_to_double(v.im); }

// ---- the sweep ------------------------------------------------------------------
// BIN: the click-number distribution mode (one pattern = all M modes): the subset
// terms are summed unsigned into bins by subset size instead of into the signed sum
template <typename T, bool BIN = false>
__global__ void __launch_bounds__(kThreads) sweep_kernel(int M, const double *__restrict__ O,
                                                        const uint64_t *__restrict__ pats, int n_pat, Plan pl) {
    using Lay = Layout<T>;
    constexpr int B = Prec<T>::B;
    extern __shared__ __align__(16) unsigned char smem[];
    T *X = (T *)(smem + Lay::off_X);
    T *Y = (T *)(smem + Lay::off_Y);
    using Node = typename Prec<T>::Node;
    using NIO = NodeIO<Node>;
    unsigned char *tauX = smem + Lay::off_tauX;
    unsigned char *tauY = smem + Lay::off_tauY;
    double *red = (double *)(smem + Lay::off_red);
    int *modes = (int *)(smem + Lay::off_modes);
    int *pos = (int *)(smem + Lay::off_pos);
    int *decoff = (int *)(smem + Lay::off_decoff);
    uint16_t *dec = (uint16_t *)(smem + Lay::off_dec);
    __shared__ long long s_unit;
    __shared__ int s_n, s_k, s_flag;
    __shared__ int s_base[kThreads];        // binned mode: modes included above each bottom node
    __shared__ typename BinOf<T>::type s_ubin[kMaxN + 1];  // binned mode: the unit's size bins
    __shared__ __align__(16) unsigned char s_vred_raw[sizeof(fx6) * (kThreads / 32)];  // fixed point: per-warp
    T *s_vred = (T *)s_vred_raw;                                                          // aligned sums
    __shared__ float s_ared[kThreads / 32];
    __shared__ int s_ered[kThreads / 32];
    T *Ub = (T *)(smem + Lay::off_U);
    T *Wb = (T *)(smem + Lay::off_W);
    T *Wpre = (T *)(smem + Lay::off_tauX);  // W rows of a prefix pivot (the prefactors are free then)
    T *Sl = (T *)(smem + Lay::off_Sl);       // the sub-unit tree's stored matrices
    using Tau = typename Prec<T>::Tau;
    __shared__ Tau s_tpre;

    const int t = threadIdx.x;
    const int N2 = 2 * M;
    // decode tables (i, j) of packed indices for every even dimension 2m <= 2R
    if (t == 0) {
        int off = 0;
        for (int m = 1; m <= Lay::R; ++m) {
            decoff[m] = off;
            off += sym(2 * m);
        }
    }
    __syncthreads();
    for (int m = 1; m <= Lay::R; ++m) {
        const int d = 2 * m;
        for (int i = t; i < d; i += kThreads)
            for (int j = i; j < d; ++j) dec[decoff[m] + pidx(d, i, j)] = (uint16_t)(i | (j << 8));
    }
    const long long total = *pl.total_units;

    for (;;) {
        if (t == 0) s_unit = (long long)atomicAdd(pl.counter, 1ull);
        __syncthreads();
        const long long u = s_unit;
        if (u >= total) break;
        // sorted pattern position: unit_off[sp] <= u < unit_off[sp + 1]
        int lo = 0, hi = n_pat;
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (pl.unit_off[mid] <= u) lo = mid; else hi = mid;
        }
        const int sp = lo;
        const int p = pl.perm[sp];
        const long long prefix = u - pl.unit_off[sp];
        const uint64_t wlo = pats[2 * p], whi = pats[2 * p + 1];
        if (t == 0) {
            int n = 0;
            for (int i = 0; i < M; ++i) {
                uint64_t w = i < 64 ? wlo : whi;
                if (w >> (i & 63) & 1ull) modes[n++] = i;
            }
            s_n = n;
            s_flag = 0;
        }
        __syncthreads();
        const int n = s_n;
        int n_eff, L_eff, q, ss;
        unit_shape<T>(n, n_eff, L_eff, q, ss, pl.split);
        const int r = L_eff + B;           // modes of a sub-unit's level-0 matrix
        const int qs = q - ss;             // prefix levels fixed by the unit index
        const int rp = ss + r;             // modes after the unit's prefix elimination
        // rows of the unit matrix: included prefix modes, then modes qs .. n_eff-1
        if (t == 0) {
            int k = 0;
            for (int a = 0; a < qs; ++a)
                if (prefix >> a & 1) pos[k++] = a;
            for (int a = qs; a < n_eff; ++a) pos[k + a - qs] = a;
            s_k = k;
        }
        __syncthreads();
        const int k = s_k;
        const int D0 = 2 * (k + rp);
        // gather G = (I - O) on those rows into X (packed; the prefix matrix spans X and Y),
        // padding modes as identity
        for (int f = t; f < (D0 >> 1) * (D0 + 1); f += kThreads) {
            int i, j;
            fold_ij(f, D0, i, j);
            const int a = pos[i >> 1], b = pos[j >> 1];
            T v;
            if (a >= n || b >= n) {
                v = konst<T>((i == j) ? 1.0 : 0.0);
            } else {
                const int si = modes[a] + (i & 1) * M, sj = modes[b] + (j & 1) * M;
                const double o = O[(size_t)si * N2 + sj];
                if (Prec<T>::fixed && !(fabs(o) <= 4.0)) atomicOr(&s_flag, 2);
                v = a_entry_t<T>(i == j ? 1.0 : 0.0, o, pl.t_re, pl.t_im);
            }
            X[pidx(D0, i, j)] = v;
        }
        __syncthreads();
        // eliminate the included prefix modes (2x2 block pivots)
        Tau tpre = Tau(1.0);
        for (int e = 0; e < k; ++e) tpre = tpre * elim_pivot<T>(X, D0, 2 * e, Wpre, &s_flag);
        // the unit's trailing 2rp x 2rp block -> Ublk, through registers: the prefix
        // matrix may extend over Ublk
        {
            const int d = 2 * rp, o = 2 * k;
            constexpr int kDm = 2 * (kS + Lay::R), kPer = (kDm * kDm + kThreads - 1) / kThreads;
            T tmp[kPer];
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                const int f = t + q * kThreads, i = f / d, j = f - (f / d) * d;
                if (f < d * d && j >= i) tmp[q] = X[pidx(D0, o + i, o + j)];
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                const int f = t + q * kThreads, i = f / d, j = f - (f / d) * d;
                if (f < d * d && j >= i) Ub[pidx(d, i, j)] = tmp[q];
            }
        }
        __syncthreads();
        const int nsub = 1 << ss;
        double u_hi = 0.0, u_lo = 0.0, u_abs = 0.0;
        fxe6 uacc6(fx6_zero(), -(1 << 20));  // fx6: the unit's sum (thread 0)
        if constexpr (BIN) {
            for (int z = t; z <= n; z += kThreads) s_ubin[z] = typename BinOf<T>::type(0.0);
        }
        // The sub-units: the include (1) / exclude (0) choices of the next ss modes of Ublk,
        // walked as a tree, depth e choosing mode e: the matrix after an include at depth e is
        // stored (in slot e + 1, or in X at the last depth), an exclude is a view of the same
        // matrix one mode further on; leaf `leaf` takes the choices of its bits from the top
        // (sub, the choice of mode e in bit e, is its bit reversal), so consecutive leaves share
        // every choice above the one that turns include.  jv[e]: the slot of the matrix the
        // node at depth e views (0: Ublk); tv[e]: the product of the includes' det^{-1/2}
        // above depth e.
        int jv[kS + 1];
        Tau tv[kS + 1];
        jv[0] = 0;
        tv[0] = Tau(1.0);
        for (int leaf = 0; leaf < nsub; ++leaf) {
            const int sub = ss ? (int)(__brev((unsigned)leaf) >> (32 - ss)) : 0;
            const int kk = __popc(sub);
            // the depth whose choice turns include (none at the first leaf); deeper
            // choices are excludes
            const int ds = leaf ? ss - 1 - (31 - __clz(leaf ^ (leaf - 1))) : ss;
            if (ds < ss) {
                const int j0 = jv[ds], D = 2 * (rp - j0);
                const T *src = j0 ? Sl + Lay::slot_off(j0) : Ub;
                T *dst = ds + 1 < ss ? Sl + Lay::slot_off(ds + 1) : X;
                const Tau rs = elim_into<T>(src, D, 2 * (ds - j0), dst, Wpre, &s_flag);
                for (int e = ds + 1; e <= ss; ++e) {
                    jv[e] = ds + 1;
                    tv[e] = tv[ds] * rs;
                }
            } else {
                for (int e = 1; e <= ss; ++e) {
                    jv[e] = 0;
                    tv[e] = Tau(1.0);
                }
            }
            const Tau tsub = tv[ss];
            // level 0 of the expansion: the leaf's matrix, packed into X (already there
            // after an include at the last depth)
            if (ds + 1 != ss) {
                const int j0 = jv[ss], D = 2 * (rp - j0), o = 2 * (ss - j0), d = 2 * r;
                const T *src = j0 ? Sl + Lay::slot_off(j0) : Ub;
                for (int f = t; f < (d >> 1) * (d + 1); f += kThreads) {
                    int i, j;
                    fold_ij(f, d, i, j);
                    X[pidx(d, i, j)] = src[pidx(D, o + i, o + j)];
                }
            }
            if (t == 0) NIO::st(tauX, 0, node_one<Node>());
            __syncthreads();
            // breadth-first expansion of L_eff levels: node c at level l + 1 is child
            // c & 1 (0 exclude, 1 include) of parent c >> 1
            for (int l = 0; l < L_eff; ++l) {
                const T *src = (l & 1) ? Y : X;
                T *dst = (l & 1) ? X : Y;
                const unsigned char *tsrc = (l & 1) ? tauY : tauX;
                unsigned char *tdst = (l & 1) ? tauX : tauY;
                T *Qb = dst;  // the parents' pivot quantities, read before the children are written
                const int d = 2 * (r - l), dc = d - 2;
                const int sstr = nstride(d), dstr = nstride(dc), Ec = sym(dc);
                const int np = 1 << l;
                // (a) the parents' pivot quantities and the children's prefactors
                if constexpr (Prec<T>::fixed) {
                    // two lanes per parent: the even lane's p00^{-1/2} and the odd lane's
                    // det^{-1/2} run side by side (whole warps, for the shuffle)
                    if (t < ((2 * np + 31) & ~31)) {
                        const int cp = min(t >> 1, np - 1), odd = t & 1;
                        const T *P = src + cp * sstr;
                        const T p00 = P[pidx(d, 0, 0)], p01 = P[pidx(d, 0, 1)], p11 = P[pidx(d, 1, 1)];
                        const T det = fx_det2(p00, p01, p11);
                        const T y = rsq<T>(odd ? det : p00);
                        const T yo = fx_shfl_xor(y, 1);
                        if (!odd && t < 2 * np) {
                            const typename Prec<T>::Piv v = fx_pivot_from(p00, p01, det, y, yo);
                            Qb[3 * cp] = v.a;
                            Qb[3 * cp + 1] = v.c;
                            Qb[3 * cp + 2] = v.b;
                            const Node tp = NIO::ld(tsrc, cp);
                            NIO::st(tdst, 2 * cp, tp);
                            NIO::st(tdst, 2 * cp + 1, node_times(tp, v.rs));
                            const int bad = fx_chol_bad(p00, det);
                            if (bad) atomicOr(&s_flag, bad);
                        }
                    }
                } else if (t < np) {
                    const T *P = src + t * sstr;
                    const T p00 = P[pidx(d, 0, 0)], p01 = P[pidx(d, 0, 1)], p11 = P[pidx(d, 1, 1)];
                    const T det = det2(p00, p01, p11);
                    const T rs = rsq<T>(det);
                    const T inv = rs * rs;
                    Qb[3 * t] = p11 * inv;
                    Qb[3 * t + 1] = -p01 * inv;
                    Qb[3 * t + 2] = p00 * inv;
                    const int bad = pivot_bad(det);
                    const Node tp = NIO::ld(tsrc, t);
                    NIO::st(tdst, 2 * t, tp);
                    NIO::st(tdst, 2 * t + 1, node_times(tp, rs));
                    if (bad) atomicOr(&s_flag, bad);
                }
                __syncthreads();
                // (b) the rows of W = B P^{-1} (fixed point: of U = B R^{-T}), dc per parent
                for (int f = t; f < np * dc; f += kThreads) {
                    const int cp = f / dc, i = f - cp * dc;
                    const T *P = src + cp * sstr;
                    const T b0 = P[pidx(d, 0, i + 2)], b1 = P[pidx(d, 1, i + 2)];
                    if constexpr (Prec<T>::fixed) {
                        const typename Prec<T>::Piv v{Qb[3 * cp], Qb[3 * cp + 1], Qb[3 * cp + 2], konst<T>(0.0),
                                                      konst<T>(0.0)};
                        fx_urow(v, b0, b1, Wb[3 * f], Wb[3 * f + 1], Wb[3 * f + 2]);
                    } else {
                        const T q00 = Qb[3 * cp], q01 = Qb[3 * cp + 1], q11 = Qb[3 * cp + 2];
                        Wb[2 * f] = dot2(q00, b0, q01, b1);
                        Wb[2 * f + 1] = dot2(q01, b0, q11, b1);
                    }
                }
                __syncthreads();
                // (c) both children of every parent: the exclude child is the parent's
                // trailing block, the include child its Schur complement
                const uint16_t *dtab = dec + decoff[dc >> 1];
                const int qstep = kThreads / Ec, rstep = kThreads - qstep * Ec;
                int cp = t / Ec, e = t - cp * Ec;
                for (int f = t; f < np * Ec; f += kThreads) {
                    const int ij = dtab[e];
                    const int i = ij & 0xff, j = ij >> 8;
                    const T *P = src + cp * sstr;
                    const T v = P[pidx(d, i + 2, j + 2)];
                    dst[(2 * cp) * dstr + e] = v;
                    if constexpr (Prec<T>::fixed) {
                        const T *Ui = Wb + 3 * (cp * dc + i), *Uj = Wb + 3 * (cp * dc + j);
                        dst[(2 * cp + 1) * dstr + e] = fx_sym_update(v, Ui[0], Ui[1], Ui[2], Uj[0], Uj[1], Uj[2]);
                    } else {
                        const T *Wr = Wb + 2 * (cp * dc + i);
                        dst[(2 * cp + 1) * dstr + e] =
                            fms2(v, Wr[0], P[pidx(d, 0, j + 2)], Wr[1], P[pidx(d, 1, j + 2)]);
                    }
                    e += rstep;
                    cp += qstep;
                    if (e >= Ec) {
                        e -= Ec;
                        ++cp;
                    }
                }
                __syncthreads();
            }
            // register-resident bottom B levels, one node per thread
            if constexpr (BIN) {
                // the thread's subtree bins (relative sizes 0..B), scaled by its prefactor,
                // then every size bin summed over the threads in a fixed order
                constexpr int NB = B + 1;
                using BT = typename BinOf<T>::type;
                BinAcc<T, NB> acc;
#pragma unroll
                for (int b = 0; b < NB; ++b) acc.v[b] = konst<T>(0.0);
                acc.bad = 0;
                BT sb[NB];
                const bool has = t < (1 << L_eff);
                if (has) {
                    const T *node = ((L_eff & 1) ? Y : X) + t * nstride(2 * B);
                    const Node tn = NIO::ld((L_eff & 1) ? tauY : tauX, t);
                    const int nreal = n - (n_eff - B);
                    SmemMat<T, B> A{node};
                    dfs<T, B, 0, false>(A, konst<T>(1.0), 0, nreal, acc, 0);
#pragma unroll
                    for (int b = 0; b < NB; ++b) sb[b] = scale_bin(tn, tsub, acc.v[b]);
                    if (node_nan(tn)) atomicOr(&s_flag, 1);
                    if (acc.bad) atomicOr(&s_flag, acc.bad);
                }
                __syncthreads();  // the nodes are read: X is scratch until the next sub-unit
                BT *tb = (BT *)X;
                if (has)
#pragma unroll
                    for (int b = 0; b < NB; ++b) tb[t * NB + b] = sb[b];
                s_base[t] = has ? k + kk + __popc(t) : -(1 << 20);
                __syncthreads();
                for (int z = t; z <= n; z += kThreads) {
                    BT sz = BT(0.0);
                    for (int t2 = 0; t2 < (1 << L_eff); ++t2) {
                        const int b = z - s_base[t2];
                        if (b >= 0 && b < NB) sz += tb[t2 * NB + b];
                    }
                    s_ubin[z] = s_ubin[z] + sz;
                }
            } else if constexpr (Prec<T>::fixed) {
                // each thread's subtree sum relative to its prefactor m 2^e, then one
                // exponent-aligned fixed-point sum over the CTA: a single conversion to
                // double-double per sub-unit
                T v = konst<T>(0.0);
                int e = -(1 << 20);
                float ab = 0.0f;
                if (t < (1 << L_eff)) {
                    const T *node = ((L_eff & 1) ? Y : X) + t * nstride(2 * B);
                    const Node tn = NIO::ld((L_eff & 1) ? tauY : tauX, t);
                    const int nreal = n - (n_eff - B);
                    Acc<T> acc{konst<T>(0.0), konst<T>(0.0), 0, 0};
                    SmemMat<T, B> A{node};
                    dfs<T, B, 0, false>(A, konst<T>(1.0), 0, nreal, acc, 0);
                    const int excl = (qs - k) + (ss - kk) + (L_eff - __popc(t));
                    v = fx_neg_if(fx_mul_su(acc.hi, tn.m), excl & 1);   // |v| < 2^11
                    e = tn.e;
                    ab = acc.abs * abs_part(tn.m);
                    if (acc.bad) atomicOr(&s_flag, acc.bad);
                }
                int em = __reduce_max_sync(0xffffffffu, e);
                if ((t & 31) == 0) s_ered[t >> 5] = em;
                __syncthreads();
                em = s_ered[0];
#pragma unroll
                for (int w = 1; w < kThreads / 32; ++w) em = max(em, s_ered[w]);
                // align to 2^(em + 4): the CTA sum of 128 terms stays below 2^14
                v = fx_shr(v, em - e + 4);
                ab = ldexpf(ab, max(e - em, -126));
#pragma unroll
                for (int off = 16; off; off >>= 1) {
                    v = v + fx_shfl_xor(v, off);
                    ab += __shfl_xor_sync(0xffffffffu, ab, off);
                }
                if ((t & 31) == 0) {
                    s_vred[t >> 5] = v;
                    s_ared[t >> 5] = ab;
                }
                __syncthreads();
                if (t == 0) {
                    T S = s_vred[0];
                    float AB = s_ared[0];
#pragma unroll
                    for (int w = 1; w < kThreads / 32; ++w) {
                        S = S + s_vred[w];
                        AB += s_ared[w];
                    }
                    if constexpr (std::is_same<T, fx6>::value) {
                        // the sub-unit's sum S 2^(em + 4) times its prefix factor, added to the
                        // unit's sum, all as m 2^e with 192-bit mantissas
                        uacc6 = fxe6_add(uacc6, fxe6_norm(S, em + 4) * tsub);
                    } else {
                        const dd sv = fx_to_dd(S);
                        const double sc = ldexp(1.0, em + 4);
                        unit_add(u_hi, u_lo, tsub, sv.hi * sc, sv.lo * sc);
                    }
                    u_abs += tau_abs(tsub) * ldexp((double)AB, em);
                }
            } else if (t < (1 << L_eff)) {
                const T *node = ((L_eff & 1) ? Y : X) + t * nstride(2 * B);
                const Node tau_node = NIO::ld((L_eff & 1) ? tauY : tauX, t);
                const int nreal = n - (n_eff - B);
                Acc<T> acc{konst<T>(0.0), konst<T>(0.0), 0, 0};
                SmemMat<T, B> A{node};
                dfs<T, B, 0, false>(A, konst<T>(1.0), 0, nreal, acc, 0);
                const int excl = (qs - k) + (ss - kk) + (L_eff - __popc(t));
                const Tau sc = Tau((excl & 1) ? -1.0 : 1.0) * Tau(tau_node) * tsub;
                double sh, sl;
                sum_parts(acc.hi, acc.lo, sh, sl);
                unit_add(u_hi, u_lo, sc, sh, sl);
                u_abs += tau_abs(sc) * to_hi(acc.abs);
                if (is_nan(acc.abs) || is_nan(tau_node)) atomicOr(&s_flag, 1);
            }
            __syncthreads();   // X / Y are rewritten by the next sub-unit
        }
        if constexpr (BIN) {
            // the unit's bins times its prefix factor (thread z owns bin z)
            double *out = pl.partials + (size_t)2 * (n + 1) * u;
            for (int z = t; z <= n; z += kThreads) {
                store2(out + 2 * z, tpre * s_ubin[z]);
            }
            if (t == 0 && (s_flag || is_nan(tpre))) atomicOr(pl.pflags + sp, 1);
            __syncthreads();
        } else if constexpr (std::is_same<T, fx6>::value) {
            // thread 0 holds the unit's whole sum: times the prefix factor, stored as the
            // 192-bit mantissa (three words), the exponent and the sum of |terms|
            if (t == 0) {
                const fxe6 r = uacc6 * tpre;
                double *out = pl.partials + (size_t)partial_words<T>() * u;
                uint32_t *mw = (uint32_t *)out;
#pragma unroll
                for (int k = 0; k < 6; ++k) mw[k] = r.m.w[k];
                out[3] = (double)r.e;
                out[4] = u_abs * tau_abs(tpre);
                if (s_flag) atomicOr(pl.pflags + sp, s_flag);
            }
            __syncthreads();
        } else {
        double c_hi = u_hi, c_lo = u_lo, c_abs = u_abs;
        // deterministic CTA reduction (TwoSum tree)
        for (int off = 16; off; off >>= 1) {
            double oh = __shfl_xor_sync(0xffffffffu, c_hi, off);
            double ol = __shfl_xor_sync(0xffffffffu, c_lo, off);
            double oa = __shfl_xor_sync(0xffffffffu, c_abs, off);
            double s, e;
            two_sum(c_hi, oh, s, e);
            c_hi = s;
            c_lo += ol + e;
            c_abs += oa;
        }
        if ((t & 31) == 0) {
            red[3 * (t >> 5)] = c_hi;
            red[3 * (t >> 5) + 1] = c_lo;
            red[3 * (t >> 5) + 2] = c_abs;
        }
        if (t == 0) s_tpre = tpre;
        __syncthreads();
        if (t == 0) {
            double h = red[0], l = red[1], a = red[2];
            for (int w = 1; w < kThreads / 32; ++w) {
                double s, e;
                two_sum(h, red[3 * w], s, e);
                h = s;
                l += red[3 * w + 1] + e;
                a += red[3 * w + 2];
            }
            const Tau tp = s_tpre;
            unit_scale(h, l, tp);
            double *out = pl.partials + 3 * u;
            out[0] = h;
            out[1] = l;
            out[2] = a * tau_hi(tp);
            const int fl = s_flag | (is_nan(tp) ? 1 : 0);
            if (fl) atomicOr(pl.pflags + sp, fl);
        }
        __syncthreads();
        }
    }
}

// ---- per-pattern result ---------------------------------------------------------------
// log P, kappa, the a-posteriori bound and the status of one pattern from its signed sum
// (h, l) and sum of |terms| a.  flags: pivot bits of its units (1 not positive, 2 outside
// the fixed-point range); n < 0: invalid pattern; over: the batch did not fit.
template <typename T>
__device__ __forceinline__ void finish_pattern(int n, bool over, int flags, double h, double l, double a,
                                               double logdet, double &lp, double &kap, double &eb, int &st) {
    const double Tv = h + l;
    st = GBS_OK;
    lp = nan("");
    kap = nan("");
    eb = nan("");
    if (n < 0) {
        st = GBS_E_INVALID;
    } else if (over) {
        st = GBS_E_NOMEM;
    } else if (flags != 0) {
        st = (flags & 1) ? GBS_E_NOT_SPD : GBS_E_RANGE;
    } else {
        // a-posteriori bound: every term carries a relative error of at most
        // c (2n + 4) u from its chain of 2x2 pivots; the signed sum amplifies by kappa.
        const double uu = Prec<T>::u;
        kap = a / fabs(Tv);
        const double rel = 4.0 * kap * (2.0 * n + 4.0) * uu + 4.0 * kap * Prec<T>::u_sum;
        if (!(Tv > 0.0)) {
            st = GBS_E_NONPOSITIVE;
        } else {
            lp = -0.5 * logdet + log(h) + log1p(l / h);
            eb = rel < 1.0 ? -log1p(-rel) : INFINITY;
        }
    }
}

// the unit partials u0 <= u < u1 of one pattern summed in unit order by one warp (lanes
// stride the units, then a fixed pairing tree: deterministic); the result on lane 0
__device__ __forceinline__ void warp_unit_sum(const double *__restrict__ partials, long long u0, long long u1,
                                              int lane, double &h, double &l, double &a) {
    h = 0.0;
    l = 0.0;
    a = 0.0;
    for (long long u = u0 + lane; u < u1; u += 32) {
        const double *q = partials + 3 * u;
        double s, e;
        two_sum(h, q[0], s, e);
        h = s;
        l += q[1] + e;
        a += q[2];
    }
    for (int off = 1; off < 32; off <<= 1) {
        double oh = __shfl_down_sync(0xffffffffu, h, off);
        double ol = __shfl_down_sync(0xffffffffu, l, off);
        double oa = __shfl_down_sync(0xffffffffu, a, off);
        if ((lane & (2 * off - 1)) == 0) {
            double s, e;
            two_sum(h, oh, s, e);
            h = s;
            l += ol + e;
            a += oa;
        }
    }
}

// ---- per-pattern result: sum of the pattern's unit partials in unit order -------------
template <typename T>
__global__ void finalize_kernel(int n_pat, const double *__restrict__ logdet, Plan pl,
                                double *__restrict__ logP, double *__restrict__ kappa,
                                double *__restrict__ err_bound, int32_t *__restrict__ status) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n_pat) return;
    const int sp = warp;
    const int p = pl.perm[sp];
    const int n = pl.pat_n[p];
    const bool batch_over = *pl.overflow != 0;
    double h, l, a;
    warp_unit_sum(pl.partials, pl.unit_off[sp], batch_over ? pl.unit_off[sp] : pl.unit_off[sp + 1], lane, h, l, a);
    if (lane) return;
    double lp, kap, eb;
    int st;
    finish_pattern<T>(n, batch_over, pl.pflags[sp], h, l, a, *logdet, lp, kap, eb, st);
    logP[p] = lp;
    if (kappa) kappa[p] = kap;
    if (err_bound) err_bound[p] = eb;
    if (status) status[p] = st;
}

// fx6: the pattern's unit sums (m 2^e, 192-bit mantissas) added in unit order by one warp,
// aligned to the larger exponent at each step (every addend loses at most its bits below
// 2^-176 of the larger), then the same result and bound as every other precision
__device__ __forceinline__ fxe6 fxe6_shfl_down(const fxe6 &a, int off) {
    fxe6 r;
#pragma unroll
    for (int k = 0; k < 6; ++k) r.m.w[k] = __shfl_down_sync(0xffffffffu, a.m.w[k], off);
    r.e = __shfl_down_sync(0xffffffffu, a.e, off);
    return r;
}
__global__ void finalize6_kernel(int n_pat, const double *__restrict__ logdet, Plan pl, double *__restrict__ logP,
                                 double *__restrict__ kappa, double *__restrict__ err_bound,
                                 int32_t *__restrict__ status) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n_pat) return;
    const int sp = warp;
    const int p = pl.perm[sp];
    const int n = pl.pat_n[p];
    const bool batch_over = *pl.overflow != 0;
    const long long u0 = pl.unit_off[sp], u1 = batch_over ? u0 : pl.unit_off[sp + 1];
    constexpr int W = partial_words<fx6>();
    fxe6 acc(fx6_zero(), -(1 << 20));
    double a = 0.0;
    for (long long u = u0 + lane; u < u1; u += 32) {
        const double *q = pl.partials + (size_t)W * u;
        const uint32_t *mw = (const uint32_t *)q;
        fxe6 v;
#pragma unroll
        for (int k = 0; k < 6; ++k) v.m.w[k] = mw[k];
        v.e = (int)q[3];
        acc = fxe6_add(acc, v);
        a += q[4];
    }
    for (int off = 1; off < 32; off <<= 1) {  // fixed pairing order: deterministic
        const fxe6 o = fxe6_shfl_down(acc, off);
        const double oa = __shfl_down_sync(0xffffffffu, a, off);
        if ((lane & (2 * off - 1)) == 0) {
            acc = fxe6_add(acc, o);
            a += oa;
        }
    }
    if (lane) return;
    double lp, kap, eb;
    int st;
    finish_pattern<fx6>(n, batch_over, pl.pflags[sp], fxe6_to_double(acc), 0.0, a, *logdet, lp, kap, eb, st);
    logP[p] = lp;
    if (kappa) kappa[p] = kap;
    if (err_bound) err_bound[p] = eb;
    if (status) status[p] = st;
}

// ---- one slice of a batch's work units (the batch split across GPUs) ------------------
// After the plan: the sweep evaluates only units [total part / nparts, total (part + 1) /
// nparts) (units of one precision and split carry equal numbers of subsets once n >= B + L
// + s, so equal unit counts balance the cost; a slice may cut a large pattern by prefix).
__global__ void slice_kernel(Plan pl, int part, int nparts, long long *range) {
    const long long total = *pl.total_units;  // 0 when the batch did not fit
    const long long b = total * part / nparts, e = total * (part + 1) / nparts;
    range[0] = b;
    range[1] = e;
    *pl.counter = (unsigned long long)b;
    *pl.total_units = e;
}

// per pattern: the slice's units of the pattern summed in unit order -> (T_hi, T_lo,
// sum |terms|) and its flags (-1 invalid pattern; else bits 1 not positive, 2 outside the
// fixed-point range, 4 the batch did not fit)
__global__ void slice_partial_kernel(int n_pat, Plan pl, const long long *__restrict__ range,
                                     double *__restrict__ part, int32_t *__restrict__ pflag) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n_pat) return;
    const int sp = warp;
    const int p = pl.perm[sp];
    const int n = pl.pat_n[p];
    const bool over = *pl.overflow != 0;
    long long u0 = pl.unit_off[sp], u1 = pl.unit_off[sp + 1];
    u0 = u0 > range[0] ? u0 : range[0];
    u1 = u1 < range[1] ? u1 : range[1];
    if (over || u1 < u0) u1 = u0;
    double h, l, a;
    warp_unit_sum(pl.partials, u0, u1, lane, h, l, a);
    if (lane) return;
    part[3 * p] = h;
    part[3 * p + 1] = l;
    part[3 * p + 2] = a;
    pflag[p] = n < 0 ? -1 : ((u1 > u0 ? pl.pflags[sp] : 0) | (over ? 4 : 0));
}

// the slices' partial sums of every pattern combined in slice order (TwoSum), then the
// result as gbs_prob's; n from the pattern's bits
template <typename T>
__global__ void combine_kernel(int n_pat, int nparts, const uint64_t *__restrict__ pats,
                               const double *__restrict__ logdet, const double *__restrict__ parts,
                               const int32_t *__restrict__ pflags, double *__restrict__ logP,
                               double *__restrict__ kappa, double *__restrict__ err_bound,
                               int32_t *__restrict__ status) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pat) return;
    double h = 0.0, l = 0.0, a = 0.0;
    int flags = 0;
    bool invalid = false;
    for (int q = 0; q < nparts; ++q) {
        const size_t i = (size_t)q * n_pat + p;
        const int f = pflags[i];
        if (f < 0) invalid = true;
        else flags |= f;
        double s, e;
        two_sum(h, parts[3 * i], s, e);
        h = s;
        l += parts[3 * i + 1] + e;
        a += parts[3 * i + 2];
    }
    const int n = invalid ? -1 : __popcll(pats[2 * p]) + __popcll(pats[2 * p + 1]);
    double lp, kap, eb;
    int st;
    finish_pattern<T>(n, (flags & 4) != 0, flags & 3, h, l, a, *logdet, lp, kap, eb, st);
    logP[p] = lp;
    if (kappa) kappa[p] = kap;
    if (err_bound) err_bound[p] = eb;
    if (status) status[p] = st;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

struct WsOffsets {
    size_t counter, total, overflow, range, perm, pat_n, unit_off, pflags, partials, end;
};

WsOffsets ws_offsets(int n_pat, long long units, int pw = 3) {
    WsOffsets o;
    o.counter = 0;
    o.total = 8;
    o.overflow = 16;
    o.range = 24;  // two long long: the unit slice of gbs_prob_partial
    o.perm = align256(40);
    o.pat_n = align256(o.perm + 4 * (size_t)n_pat);
    o.unit_off = align256(o.pat_n + 4 * (size_t)n_pat);
    o.pflags = align256(o.unit_off + 8 * ((size_t)n_pat + 1));
    o.partials = align256(o.pflags + 4 * (size_t)n_pat);
    o.end = o.partials + 8 * (size_t)pw * (size_t)units;
    return o;
}

Plan plan_from(void *ws, int n_pat) {
    WsOffsets o = ws_offsets(n_pat, 0);
    char *b = (char *)ws;
    Plan pl;
    pl.counter = (unsigned long long *)(b + o.counter);
    pl.total_units = (long long *)(b + o.total);
    pl.overflow = (int *)(b + o.overflow);
    pl.perm = (int *)(b + o.perm);
    pl.pat_n = (int *)(b + o.pat_n);
    pl.unit_off = (long long *)(b + o.unit_off);
    pl.pflags = (int *)(b + o.pflags);
    pl.partials = (double *)(b + o.partials);
    pl.split = kS;
    pl.t_re = 0.0;
    pl.t_im = 0.0;
    return pl;
}

template <typename T>
int run_sweep(gbs_ctx *ctx, int M, const double *O, const double *logdet, const uint64_t *pats,
              int n_pat, double *logP, double *kappa, double *err_bound, int32_t *status) {
    using Lay = Layout<T>;
    const int pi = Prec<T>::idx;
    if (ctx->reserved && n_pat > ctx->cap_pat)
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_prob: %d patterns exceed the reservation of %d",
                        n_pat, ctx->cap_pat);
    if (ctx->sweep_blocks_per_sm[pi] == 0) {
        GBS_CUDA(ctx, cudaFuncSetAttribute(sweep_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)Lay::bytes));
        int nb = 0;
        GBS_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<T>, kThreads,
                                                                    Lay::bytes));
        if (nb < 1) return gbs_fail(ctx, GBS_E_CUDA, "sweep kernel does not fit on an SM");
        ctx->sweep_blocks_per_sm[pi] = nb;
    }
    long long cap;
    if (ctx->reserved) {
        cap = (long long)((ctx->ws_bytes - ws_offsets(n_pat, 0).partials) / (8 * partial_words<T>()));
    } else {
        int st = gbs_ws_ensure(ctx, ws_offsets(n_pat, 0).end);
        if (st) return st;
        cap = (long long)((ctx->ws_bytes - ws_offsets(n_pat, 0).partials) / (8 * partial_words<T>()));
    }
    Plan pl = plan_from(ctx->ws, n_pat);
    pl.split = sweep_split_of(ctx, pi);
    plan_kernel<T><<<1, kPlanThreads, 0, ctx->stream>>>(M, pats, n_pat, cap, pl);
    GBS_CUDA(ctx, cudaGetLastError());
    if (!ctx->reserved) {
        // size the unit partials: one small readback
        GBS_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, pl.unit_off + n_pat, 8, cudaMemcpyDeviceToHost,
                                      ctx->stream));
        GBS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        long long need = *(long long *)ctx->pinned;
        if (need > cap) {
            int st = gbs_ws_ensure(ctx, ws_offsets(n_pat, need, partial_words<T>()).end);
            if (st) return st;
            cap = (long long)((ctx->ws_bytes - ws_offsets(n_pat, 0).partials) / (8 * partial_words<T>()));
            pl = plan_from(ctx->ws, n_pat);
            pl.split = sweep_split_of(ctx, pi);
            plan_kernel<T><<<1, kPlanThreads, 0, ctx->stream>>>(M, pats, n_pat, cap, pl);
            GBS_CUDA(ctx, cudaGetLastError());
        }
    }
    const int grid = ctx->num_sms * ctx->sweep_blocks_per_sm[pi];
    int st = gbs_timing_begin(ctx);
    if (st) return st;
    sweep_kernel<T><<<grid, kThreads, Lay::bytes, ctx->stream>>>(M, O, pats, n_pat, pl);
    GBS_CUDA(ctx, cudaGetLastError());
    st = gbs_timing_end(ctx);
    if (st) return st;
    const int fthreads = 256, fblocks = (n_pat * 32 + fthreads - 1) / fthreads;
    if constexpr (std::is_same<T, fx6>::value)
        finalize6_kernel<<<fblocks, fthreads, 0, ctx->stream>>>(n_pat, logdet, pl, logP, kappa, err_bound, status);
    else
        finalize_kernel<T><<<fblocks, fthreads, 0, ctx->stream>>>(n_pat, logdet, pl, logP, kappa,
                                                                 err_bound, status);
    GBS_CUDA(ctx, cudaGetLastError());
    return GBS_OK;
}

// The same launch sequence on a workspace the caller provides: no allocation,
// no synchronisation.  A batch whose units do not fit reports GBS_E_NOMEM per pattern.
template <typename T>
int run_sweep_on(gbs_ctx *ctx, void *ws, size_t ws_bytes, int M, const double *O,
                 const double *logdet, const uint64_t *pats, int n_pat, double *logP,
                 double *kappa, double *err_bound, int32_t *status) {
    using Lay = Layout<T>;
    const int pi = Prec<T>::idx;
    if (ctx->sweep_blocks_per_sm[pi] == 0) {
        GBS_CUDA(ctx, cudaFuncSetAttribute(sweep_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)Lay::bytes));
        int nb = 0;
        GBS_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<T>, kThreads,
                                                                    Lay::bytes));
        if (nb < 1) return gbs_fail(ctx, GBS_E_CUDA, "sweep kernel does not fit on an SM");
        ctx->sweep_blocks_per_sm[pi] = nb;
    }
    const size_t base = ws_offsets(n_pat, 0).partials;
    if (ws_bytes < base)
        return gbs_fail(ctx, GBS_E_INVALID, "workspace of %zu bytes cannot hold %d patterns", ws_bytes, n_pat);
    const long long cap = (long long)((ws_bytes - base) / 24);
    Plan pl = plan_from(ws, n_pat);
    pl.split = sweep_split_of(ctx, pi);
    plan_kernel<T><<<1, kPlanThreads, 0, ctx->stream>>>(M, pats, n_pat, cap, pl);
    GBS_CUDA(ctx, cudaGetLastError());
    const int grid = ctx->num_sms * ctx->sweep_blocks_per_sm[pi];
    sweep_kernel<T><<<grid, kThreads, Lay::bytes, ctx->stream>>>(M, O, pats, n_pat, pl);
    GBS_CUDA(ctx, cudaGetLastError());
    const int fthreads = 256, fblocks = (n_pat * 32 + fthreads - 1) / fthreads;
    finalize_kernel<T><<<fblocks, fthreads, 0, ctx->stream>>>(n_pat, logdet, pl, logP, kappa,
                                                             err_bound, status);
    GBS_CUDA(ctx, cudaGetLastError());
    return GBS_OK;
}

// One slice of the batch's work units (gbs_prob_partial): the plan of the whole batch,
// then only this slice's units swept, and per-pattern partial sums of the slice.
template <typename T>
int run_sweep_slice(gbs_ctx *ctx, int M, const double *O, const uint64_t *pats, int n_pat, int part,
                    int nparts, double *partial, int32_t *pflag) {
    using Lay = Layout<T>;
    const int pi = Prec<T>::idx;
    if (ctx->reserved && n_pat > ctx->cap_pat)
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_prob_partial: %d patterns exceed the reservation of %d",
                        n_pat, ctx->cap_pat);
    if (ctx->sweep_blocks_per_sm[pi] == 0) {
        GBS_CUDA(ctx, cudaFuncSetAttribute(sweep_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)Lay::bytes));
        int nb = 0;
        GBS_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<T>, kThreads,
                                                                    Lay::bytes));
        if (nb < 1) return gbs_fail(ctx, GBS_E_CUDA, "sweep kernel does not fit on an SM");
        ctx->sweep_blocks_per_sm[pi] = nb;
    }
    if (!ctx->reserved) {
        int st = gbs_ws_ensure(ctx, ws_offsets(n_pat, 0).end);
        if (st) return st;
    }
    long long cap = (long long)((ctx->ws_bytes - ws_offsets(n_pat, 0).partials) / 24);
    Plan pl = plan_from(ctx->ws, n_pat);
    pl.split = sweep_split_of(ctx, pi);
    plan_kernel<T><<<1, kPlanThreads, 0, ctx->stream>>>(M, pats, n_pat, cap, pl);
    GBS_CUDA(ctx, cudaGetLastError());
    if (!ctx->reserved) {
        GBS_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, pl.unit_off + n_pat, 8, cudaMemcpyDeviceToHost, ctx->stream));
        GBS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        const long long need = *(long long *)ctx->pinned;
        if (need > cap) {
            int st = gbs_ws_ensure(ctx, ws_offsets(n_pat, need).end);
            if (st) return st;
            cap = (long long)((ctx->ws_bytes - ws_offsets(n_pat, 0).partials) / 24);
            pl = plan_from(ctx->ws, n_pat);
            pl.split = sweep_split_of(ctx, pi);
            plan_kernel<T><<<1, kPlanThreads, 0, ctx->stream>>>(M, pats, n_pat, cap, pl);
            GBS_CUDA(ctx, cudaGetLastError());
        }
    }
    long long *range = (long long *)((char *)ctx->ws + ws_offsets(n_pat, 0).range);
    slice_kernel<<<1, 1, 0, ctx->stream>>>(pl, part, nparts, range);
    GBS_CUDA(ctx, cudaGetLastError());
    const int grid = ctx->num_sms * ctx->sweep_blocks_per_sm[pi];
    int st = gbs_timing_begin(ctx);
    if (st) return st;
    sweep_kernel<T><<<grid, kThreads, Lay::bytes, ctx->stream>>>(M, O, pats, n_pat, pl);
    GBS_CUDA(ctx, cudaGetLastError());
    st = gbs_timing_end(ctx);
    if (st) return st;
    const int fthreads = 256, fblocks = (n_pat * 32 + fthreads - 1) / fthreads;
    slice_partial_kernel<<<fblocks, fthreads, 0, ctx->stream>>>(n_pat, pl, range, partial, pflag);
    GBS_CUDA(ctx, cudaGetLastError());
    return GBS_OK;
}

// ---- click-number distribution: bins of all subsets of the M modes by size ----------
__global__ void all_modes_kernel(int M, uint64_t *pat) {
    pat[0] = M >= 64 ? ~0ull : ((1ull << M) - 1);
    pat[1] = M > 64 ? (M >= 128 ? ~0ull : ((1ull << (M - 64)) - 1)) : 0ull;
}

// per chunk of 1024 units: every size bin summed in unit order
__global__ void bins_chunk_kernel(int nb, const double *__restrict__ partials, const long long *__restrict__ units_p,
                                  double *__restrict__ chunks) {
    const long long c = blockIdx.x, units = *units_p;
    const long long u0 = c * 1024, u1 = (c + 1) * 1024 < units ? (c + 1) * 1024 : units;
    for (int z = threadIdx.x; z < nb; z += blockDim.x) {
        dd acc = dd(0.0);
        for (long long u = u0; u < u1; ++u)
            acc += dd(partials[(size_t)2 * nb * u + 2 * z], partials[(size_t)2 * nb * u + 2 * z + 1]);
        chunks[(size_t)2 * nb * c + 2 * z] = acc.hi;
        chunks[(size_t)2 * nb * c + 2 * z + 1] = acc.lo;
    }
}

// E_z = sum_{|Z| = z} det(A_Z)^{-1/2} from the chunks, then
//   p(n) = det(sigma_Q)^{-1/2} sum_{z <= n} (-1)^{n - z} C(M - z, n - z) E_z
// (every pattern S with n clicks contains the subset Z in C(M - z, n - z) ways), in
// double-double with exact binomials; kappa_n = sum_z C E_z / |S_n|
__global__ void bins_final_kernel(int M, long long nchunks, const double *__restrict__ chunks,
                                  const double *__restrict__ logdet, const int *__restrict__ pflags,
                                  const int *__restrict__ overflow, double *__restrict__ logp,
                                  double *__restrict__ kappa) {
    __shared__ dd E[kMaxN + 1];
    __shared__ double Cb[kMaxN + 1][kMaxN + 1];
    const int t = threadIdx.x, nb = M + 1;
    for (int z = t; z < nb; z += blockDim.x) {
        dd acc = dd(0.0);
        for (long long c = 0; c < nchunks; ++c)
            acc += dd(chunks[(size_t)2 * nb * c + 2 * z], chunks[(size_t)2 * nb * c + 2 * z + 1]);
        E[z] = acc;
    }
    for (int a = t; a <= M; a += blockDim.x) {
        Cb[a][0] = 1.0;
        for (int b = 1; b <= a; ++b) Cb[a][b] = Cb[a][b - 1] * (double)(a - b + 1) / (double)b;  // exact below 2^53
    }
    __syncthreads();
    const bool bad = *overflow || pflags[0];
    for (int n = t; n <= M; n += blockDim.x) {
        dd S = dd(0.0);
        double A = 0.0;
        for (int z = 0; z <= n; ++z) {
            const double c = Cb[M - z][n - z];
            const dd term = dd(c) * E[z];
            S = ((n - z) & 1) ? S - term : S + term;
            A += c * fabs(E[z].hi);
        }
        const bool ok = !bad && S.hi > 0.0;
        logp[n] = ok ? -0.5 * (*logdet) + log(S.hi) + log1p(S.lo / S.hi) : nan("");
        if (kappa) kappa[n] = bad ? nan("") : A / fabs(S.hi);
    }
}

// ---- sector-resolved distribution: complex bins at one t, then the DFT over t ---------
// per chunk of 1024 units: every size bin's complex sum in unit order (double-double parts)
__global__ void zbins_chunk_kernel(int nb, const double *__restrict__ partials, const long long *__restrict__ units_p,
                                   double *__restrict__ chunks) {
    const long long c = blockIdx.x, units = *units_p;
    const long long u0 = c * 1024, u1 = (c + 1) * 1024 < units ? (c + 1) * 1024 : units;
    for (int z = threadIdx.x; z < nb; z += blockDim.x) {
        dd re = dd(0.0), im = dd(0.0);
        for (long long u = u0; u < u1; ++u) {
            re += dd(partials[(size_t)2 * nb * u + 2 * z]);
            im += dd(partials[(size_t)2 * nb * u + 2 * z + 1]);
        }
        double *o = chunks + (size_t)4 * nb * c + 4 * z;
        o[0] = re.hi;
        o[1] = re.lo;
        o[2] = im.hi;
        o[3] = im.lo;
    }
}

// G_n(t) = det(sigma_Q)^{-1/2} sum_{z <= n} (-1)^{n - z} C(M - z, n - z) E_z(t) for one t,
// E_z(t) = sum_{|Z| = z} det(I - t O_Z)^{-1/2}: the generating function of the sectors of
// the n-click probability, sum_k p_k(n) t^k.  Real and imaginary parts in double-double.
__global__ void zbins_final_kernel(int M, long long nchunks, const double *__restrict__ chunks,
                                   const double *__restrict__ logdet, const int *__restrict__ pflags,
                                   const int *__restrict__ overflow, double *__restrict__ G, int *__restrict__ bad) {
    __shared__ dd Er[kMaxN + 1], Ei[kMaxN + 1];
    __shared__ double Cb[kMaxN + 1][kMaxN + 1];
    const int t = threadIdx.x, nb = M + 1;
    for (int z = t; z < nb; z += blockDim.x) {
        dd re = dd(0.0), im = dd(0.0);
        for (long long c = 0; c < nchunks; ++c) {
            const double *o = chunks + (size_t)4 * nb * c + 4 * z;
            re += dd(o[0], o[1]);
            im += dd(o[2], o[3]);
        }
        Er[z] = re;
        Ei[z] = im;
    }
    for (int a = t; a <= M; a += blockDim.x) {
        Cb[a][0] = 1.0;
        for (int b = 1; b <= a; ++b) Cb[a][b] = Cb[a][b - 1] * (double)(a - b + 1) / (double)b;  // exact below 2^53
    }
    __syncthreads();
    const double sc = exp(-0.5 * (*logdet));
    for (int n = t; n <= M; n += blockDim.x) {
        dd Sr = dd(0.0), Si = dd(0.0);
        for (int z = 0; z <= n; ++z) {
            const dd c = dd(Cb[M - z][n - z]);
            if ((n - z) & 1) {
                Sr -= c * Er[z];
                Si -= c * Ei[z];
            } else {
                Sr += c * Er[z];
                Si += c * Ei[z];
            }
        }
        G[2 * n] = sc * Sr.hi;
        G[2 * n + 1] = sc * Si.hi;
    }
    if (t == 0 && (*overflow || pflags[0])) *bad = 1;
}

// even sectors only: G_j = conj G_{L/2 - j} for the points j = jmax + 1..h not swept
__global__ void mirror_kernel(int nb, int h, int jmax, double *__restrict__ G) {
    const int j = jmax + 1 + blockIdx.x;
    for (int n = threadIdx.x; n < nb; n += blockDim.x) {
        G[2 * nb * j + 2 * n] = G[2 * nb * (h - j) + 2 * n];
        G[2 * nb * j + 2 * n + 1] = -G[2 * nb * (h - j) + 2 * n + 1];
    }
}

// p_k(n) = rho^-k / L sum_{j < L} G_n(t_j) e^{-2 pi i j k / L}, t_j = rho e^{2 pi i j / L}, from
// j = 0..L/2 (the coefficients are real: G_n(t_{L-j}) is the conjugate of G_n(t_j));
// one thread per (k, n), row k of pkn holds p_k(0..M)
__global__ void sector_dft_kernel(int M, int L, double rho, int K, const double *__restrict__ G,
                                  const int *__restrict__ bad, double *__restrict__ pkn) {
    const int nb = M + 1;
    const long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= (long long)(K + 1) * nb) return;
    const int k = (int)(f / nb), n = (int)(f - (long long)k * nb);
    const int h = L / 2;
    double s = G[2 * n] + ((k & 1) ? -G[2 * nb * h + 2 * n] : G[2 * nb * h + 2 * n]);
    for (int j = 1; j < h; ++j) {
        double sn, cs;
        sincospi(2.0 * (double)(((long long)j * k) % L) / (double)L, &sn, &cs);
        const double gr = G[2 * nb * j + 2 * n], gi = G[2 * nb * j + 2 * n + 1];
        s += 2.0 * (gr * cs + gi * sn);  // 2 Re(G e^{-i theta})
    }
    pkn[f] = *bad ? nan("") : s / (double)L * pow(rho, -(double)k);
}

// GBS_AUTO: the patterns the fixed-point pass flagged out of range, the others replaced by a
// pattern no plan accepts (every bit set: a detector >= M, or more than kMaxN clicks)
__global__ void auto_mark_kernel(int n_pat, const int32_t *__restrict__ st, const uint64_t *__restrict__ pats,
                                 uint64_t *__restrict__ redo) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pat) return;
    const bool again = st[p] == GBS_E_RANGE;
    redo[2 * p] = again ? pats[2 * p] : ~0ull;
    redo[2 * p + 1] = again ? pats[2 * p + 1] : ~0ull;
}
// ... and the double-double results in their places
// (st and status may be the same array: each thread reads its entry before it writes it)
__global__ void auto_merge_kernel(int n_pat, const int32_t *st, const double *__restrict__ lp2,
                                  const double *__restrict__ ka2, const double *__restrict__ er2,
                                  const int32_t *__restrict__ st2, double *__restrict__ logP, double *__restrict__ kappa,
                                  double *__restrict__ err_bound, int32_t *status) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pat || st[p] != GBS_E_RANGE) return;
    logP[p] = lp2[p];
    if (kappa) kappa[p] = ka2[p];
    if (err_bound) err_bound[p] = er2[p];
    if (status) status[p] = st2[p];
}

// GBS_AUTO, last step: the patterns whose result is valid but whose bound exceeds tol (the
// sum cancels beyond 128-bit fixed point and double-double) go to the 192-bit sweep ...
__global__ void auto_mark_wide_kernel(int n_pat, const int32_t *__restrict__ st, const double *__restrict__ eb,
                                      double tol, const uint64_t *__restrict__ pats, uint64_t *__restrict__ redo) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pat) return;
    const bool again = st[p] == GBS_OK && !(eb[p] <= tol);
    redo[2 * p] = again ? pats[2 * p] : ~0ull;
    redo[2 * p + 1] = again ? pats[2 * p + 1] : ~0ull;
}
// ... and its results replace those where it succeeded
__global__ void auto_merge_wide_kernel(int n_pat, double tol, const double *__restrict__ lp3,
                                       const double *__restrict__ ka3, const double *__restrict__ er3,
                                       const int32_t *__restrict__ st3, int32_t *__restrict__ st,
                                       double *__restrict__ logP, double *__restrict__ kappa,
                                       double *__restrict__ eb) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pat) return;
    const bool again = st[p] == GBS_OK && !(eb[p] <= tol);
    if (!again || st3[p] != GBS_OK) return;
    logP[p] = lp3[p];
    kappa[p] = ka3[p];
    eb[p] = er3[p];
}

}  // namespace

size_t sweep_auto_bytes(int n_pat) {
    const size_t n = (size_t)n_pat;
    return align256(16 * n) + 5 * align256(8 * n) + 2 * align256(4 * n);
}

size_t sweep_workspace_bytes_prec(int n_pat, long long units, int precision) {
    return ws_offsets(n_pat, units, precision == GBS_FX192 ? partial_words<fx6>() : 3).end;
}

int sweep_auto(gbs_ctx *ctx, int M, const double *O, const double *logdet, const uint64_t *patterns, int n_pat,
               double *logP, double *kappa, double *err_bound, int32_t *status) {
    const size_t need = sweep_auto_bytes(n_pat);
    if (need > ctx->aux_bytes) {
        if (ctx->reserved)
            return gbs_fail(ctx, GBS_E_INVALID, "gbs_prob: %d patterns exceed the reservation of %d", n_pat,
                            ctx->cap_pat);
        GBS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (ctx->aux) GBS_CUDA(ctx, cudaFree(ctx->aux));
        ctx->aux = nullptr;
        ctx->aux_bytes = 0;
        if (cudaMalloc(&ctx->aux, need) != cudaSuccess) {
            cudaGetLastError();
            return gbs_fail(ctx, GBS_E_NOMEM, "gbs_prob: %zu bytes for the automatic precision", need);
        }
        ctx->aux_bytes = need;
    }
    const size_t n = (size_t)n_pat;
    char *b = (char *)ctx->aux;
    uint64_t *redo = (uint64_t *)b;
    double *lp2 = (double *)(b + align256(16 * n));
    double *ka2 = lp2 + align256(8 * n) / 8, *er2 = ka2 + align256(8 * n) / 8;
    double *ka1 = kappa ? kappa : er2 + align256(8 * n) / 8;
    double *eb1 = err_bound ? err_bound : er2 + 2 * (align256(8 * n) / 8);
    int32_t *st2 = (int32_t *)(er2 + 3 * (align256(8 * n) / 8));
    int32_t *st1 = status ? status : st2 + align256(4 * n) / 4;
    // 128-bit fixed point
    int r = sweep_exact(ctx, M, O, logdet, patterns, n_pat, GBS_FX, logP, ka1, eb1, st1);
    if (r) return r;
    // double-double for the patterns outside the fixed-point range
    const unsigned g = (unsigned)((n_pat + 255) / 256);
    auto_mark_kernel<<<g, 256, 0, ctx->stream>>>(n_pat, st1, patterns, redo);
    GBS_CUDA(ctx, cudaGetLastError());
    r = sweep_exact(ctx, M, O, logdet, redo, n_pat, GBS_DD, lp2, ka2, er2, st2);
    if (r) return r;
    auto_merge_kernel<<<g, 256, 0, ctx->stream>>>(n_pat, st1, lp2, ka2, er2, st2, logP, ka1, eb1, st1);
    GBS_CUDA(ctx, cudaGetLastError());
    // 192-bit fixed point for the valid results whose bound exceeds 1e-10
    constexpr double kAutoTol = 1e-10;
    auto_mark_wide_kernel<<<g, 256, 0, ctx->stream>>>(n_pat, st1, eb1, kAutoTol, patterns, redo);
    GBS_CUDA(ctx, cudaGetLastError());
    r = sweep_exact(ctx, M, O, logdet, redo, n_pat, GBS_FX192, lp2, ka2, er2, st2);
    if (r) return r;
    auto_merge_wide_kernel<<<g, 256, 0, ctx->stream>>>(n_pat, kAutoTol, lp2, ka2, er2, st2, st1, logP, ka1, eb1);
    GBS_CUDA(ctx, cudaGetLastError());
    return GBS_OK;
}

int sweep_exact_on(gbs_ctx *ctx, void *ws, size_t ws_bytes, int M, const double *O,
                   const double *logdet, const uint64_t *patterns, int n_pat, int precision,
                   double *logP, double *kappa, double *err_bound, int32_t *status) {
    if (precision == GBS_FP64)
        return run_sweep_on<double>(ctx, ws, ws_bytes, M, O, logdet, patterns, n_pat, logP, kappa,
                                    err_bound, status);
    if (precision == GBS_DD)
        return run_sweep_on<dd>(ctx, ws, ws_bytes, M, O, logdet, patterns, n_pat, logP, kappa,
                                err_bound, status);
    if (precision == GBS_FX)
        return run_sweep_on<fx>(ctx, ws, ws_bytes, M, O, logdet, patterns, n_pat, logP, kappa,
                                err_bound, status);
    return run_sweep_on<float>(ctx, ws, ws_bytes, M, O, logdet, patterns, n_pat, logP, kappa,
                               err_bound, status);
}

size_t sweep_workspace_bytes(int n_pat, long long units) { return ws_offsets(n_pat, units).end; }

int sweep_split_of(const gbs_ctx *ctx, int precision) {
    const int v = ctx->sweep_split[precision & 7];
    return v < 0 || v > kS ? kS : v;
}

long long sweep_units_upper_bound(int n_pat, int n_max, int precision, int split) {
    int n_eff, L_eff, q, ss;
    if (precision == GBS_FP64) unit_shape<double>(n_max, n_eff, L_eff, q, ss, split);
    else if (precision == GBS_DD) unit_shape<dd>(n_max, n_eff, L_eff, q, ss, split);
    else if (precision == GBS_FX) unit_shape<fx>(n_max, n_eff, L_eff, q, ss, split);
    else if (precision == GBS_FX192) unit_shape<fx6>(n_max, n_eff, L_eff, q, ss, split);
    else unit_shape<float>(n_max, n_eff, L_eff, q, ss, split);
    return (long long)n_pat << (q - ss);
}

int sweep_exact(gbs_ctx *ctx, int M, const double *O, const double *logdet,
                const uint64_t *patterns, int n_pat, int precision, double *logP, double *kappa,
                double *err_bound, int32_t *status) {
    if (precision == GBS_FP64)
        return run_sweep<double>(ctx, M, O, logdet, patterns, n_pat, logP, kappa, err_bound, status);
    if (precision == GBS_DD)
        return run_sweep<dd>(ctx, M, O, logdet, patterns, n_pat, logP, kappa, err_bound, status);
    if (precision == GBS_FX)
        return run_sweep<fx>(ctx, M, O, logdet, patterns, n_pat, logP, kappa, err_bound, status);
    if (precision == GBS_FX192)
        return run_sweep<fx6>(ctx, M, O, logdet, patterns, n_pat, logP, kappa, err_bound, status);
    return run_sweep<float>(ctx, M, O, logdet, patterns, n_pat, logP, kappa, err_bound, status);
}

int sweep_slice(gbs_ctx *ctx, int M, const double *O, const uint64_t *patterns, int n_pat, int precision,
                int part, int nparts, double *partial, int32_t *pflag) {
    if (precision == GBS_FP64)
        return run_sweep_slice<double>(ctx, M, O, patterns, n_pat, part, nparts, partial, pflag);
    if (precision == GBS_DD)
        return run_sweep_slice<dd>(ctx, M, O, patterns, n_pat, part, nparts, partial, pflag);
    if (precision == GBS_FX)
        return run_sweep_slice<fx>(ctx, M, O, patterns, n_pat, part, nparts, partial, pflag);
    return run_sweep_slice<float>(ctx, M, O, patterns, n_pat, part, nparts, partial, pflag);
}

int sweep_combine(gbs_ctx *ctx, const double *logdet, const uint64_t *patterns, int n_pat, int precision,
                  int nparts, const double *partials, const int32_t *pflags, double *logP, double *kappa,
                  double *err_bound, int32_t *status) {
    const unsigned g = (unsigned)((n_pat + 127) / 128);
    if (precision == GBS_FP64)
        combine_kernel<double><<<g, 128, 0, ctx->stream>>>(n_pat, nparts, patterns, logdet, partials, pflags,
                                                             logP, kappa, err_bound, status);
    else if (precision == GBS_DD)
        combine_kernel<dd><<<g, 128, 0, ctx->stream>>>(n_pat, nparts, patterns, logdet, partials, pflags, logP,
                                                         kappa, err_bound, status);
    else if (precision == GBS_FX)
        combine_kernel<fx><<<g, 128, 0, ctx->stream>>>(n_pat, nparts, patterns, logdet, partials, pflags, logP,
                                                         kappa, err_bound, status);
    else
        combine_kernel<float><<<g, 128, 0, ctx->stream>>>(n_pat, nparts, patterns, logdet, partials, pflags,
                                                            logP, kappa, err_bound, status);
    GBS_CUDA(ctx, cudaGetLastError());
    return GBS_OK;
}

namespace {
constexpr int kRetryInDD = -1;

// the binned sweep in T: fixed point first (flagged out of range -> kRetryInDD, read back:
// the whole device's distribution is one result), double-double otherwise
template <typename T>
int click_distribution_in(gbs_ctx *ctx, int M, const double *O, const double *logdet, double *logp,
                          double *kappa) {
    using Lay = Layout<T>;
    const int pi = Prec<T>::idx;
    const int split = sweep_split_of(ctx, pi);
    const long long units = sweep_units_upper_bound(1, M, pi, split);
    const int nb = M + 1;
    const long long nch = (units + 1023) / 1024;
    const WsOffsets o = ws_offsets(1, 0);
    const size_t off_ch = align256(o.partials + (size_t)16 * nb * units);
    const size_t off_pat = align256(off_ch + (size_t)16 * nb * nch);
    int st = gbs_ws_ensure(ctx, off_pat + 16);
    if (st) return st;
    Plan pl = plan_from(ctx->ws, 1);
    pl.split = split;
    double *chunks = (double *)((char *)ctx->ws + off_ch);
    uint64_t *pat = (uint64_t *)((char *)ctx->ws + off_pat);
    all_modes_kernel<<<1, 1, 0, ctx->stream>>>(M, pat);
    plan_kernel<T><<<1, kPlanThreads, 0, ctx->stream>>>(M, pat, 1, units, pl);
    GBS_CUDA(ctx, cudaGetLastError());
    GBS_CUDA(ctx, cudaFuncSetAttribute(sweep_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)Lay::bytes));
    int nbk = 0;
    GBS_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nbk, sweep_kernel<T, true>, kThreads, Lay::bytes));
    if (nbk < 1) return gbs_fail(ctx, GBS_E_CUDA, "binned sweep kernel does not fit on an SM");
    st = gbs_timing_begin(ctx);
    if (st) return st;
    sweep_kernel<T, true><<<ctx->num_sms * nbk, kThreads, Lay::bytes, ctx->stream>>>(M, O, pat, 1, pl);
    GBS_CUDA(ctx, cudaGetLastError());
    st = gbs_timing_end(ctx);
    if (st) return st;
    if (Prec<T>::fixed) {
        GBS_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, pl.pflags, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        GBS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (*(int *)ctx->pinned) return kRetryInDD;
    }
    bins_chunk_kernel<<<(unsigned)nch, 64, 0, ctx->stream>>>(nb, pl.partials, pl.unit_off + 1, chunks);
    bins_final_kernel<<<1, 64, 0, ctx->stream>>>(M, nch, chunks, logdet, pl.pflags, pl.overflow, logp, kappa);
    GBS_CUDA(ctx, cudaGetLastError());
    return GBS_OK;
}
}  // namespace

int click_distribution(gbs_ctx *ctx, int M, const double *O, const double *logdet, double *logp,
                       double *kappa) {
    if (M < 4 || M > kMaxDevice)
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_click_distribution: M = %d outside 4..%d", M, kMaxDevice);
    const int r = click_distribution_in<fx>(ctx, M, O, logdet, logp, kappa);
    return r == kRetryInDD ? click_distribution_in<dd>(ctx, M, O, logdet, logp, kappa) : r;
}

namespace {
template <typename T>
int sector_distribution_in(gbs_ctx *ctx, int M, const double *O, const double *logdet, int L, double rho, int K,
                           int even, double *pkn) {
    using Lay = Layout<T>;
    if (M < 4 || M > kMaxDevice)
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_sector_distribution: M = %d outside 4..%d", M, kMaxDevice);
    if (L < 4 || L > 4096 || (L & (L - 1)))
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_sector_distribution: L = %d is not a power of two in 4..4096", L);
    if (!(rho > 0.0 && rho <= 1.0))
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_sector_distribution: rho = %g outside (0, 1]", rho);
    if (K < 0 || K >= L)
        return gbs_fail(ctx, GBS_E_INVALID, "gbs_sector_distribution: K = %d outside 0..L-1", K);
    int n_eff, L_eff, q, ss;
    unit_shape<T>(M, n_eff, L_eff, q, ss, kS);
    const long long units = 1ll << (q - ss);
    const int nb = M + 1, h = L / 2;
    const long long nch = (units + 1023) / 1024;
    const WsOffsets o = ws_offsets(1, 0);
    const size_t off_ch = align256(o.partials + (size_t)16 * nb * units);
    const size_t off_pat = align256(off_ch + (size_t)32 * nb * nch);
    const size_t off_G = align256(off_pat + 16);
    const size_t off_bad = align256(off_G + (size_t)16 * nb * (h + 1));
    int st = gbs_ws_ensure(ctx, off_bad + 16);
    if (st) return st;
    Plan pl = plan_from(ctx->ws, 1);
    pl.split = kS;
    double *chunks = (double *)((char *)ctx->ws + off_ch);
    uint64_t *pat = (uint64_t *)((char *)ctx->ws + off_pat);
    double *G = (double *)((char *)ctx->ws + off_G);
    int *bad = (int *)((char *)ctx->ws + off_bad);
    GBS_CUDA(ctx, cudaFuncSetAttribute(sweep_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)Lay::bytes));
    int nbk = 0;
    GBS_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nbk, sweep_kernel<T, true>, kThreads, Lay::bytes));
    if (nbk < 1) return gbs_fail(ctx, GBS_E_CUDA, "complex binned sweep kernel does not fit on an SM");
    all_modes_kernel<<<1, 1, 0, ctx->stream>>>(M, pat);
    GBS_CUDA(ctx, cudaMemsetAsync(bad, 0, sizeof(int), ctx->stream));
    // only even sectors (G_n(-t) = G_n(t)): G at t_{j + L/2} = -t_j repeats t_j, so the
    // points j = 0..L/4 give the rest, G_j = conj G_{L/2 - j} for L/4 < j <= L/2
    const int jmax = even ? L / 4 : h;
    for (int j = 0; j <= jmax; ++j) {
        const double ang = 2.0 * 3.14159265358979323846 * (double)j / (double)L;
        pl.t_re = rho * cos(ang);
        pl.t_im = rho * sin(ang);
        plan_kernel<T><<<1, kPlanThreads, 0, ctx->stream>>>(M, pat, 1, units, pl);
        GBS_CUDA(ctx, cudaGetLastError());
        st = gbs_timing_begin(ctx);
        if (st) return st;
        sweep_kernel<T, true><<<ctx->num_sms * nbk, kThreads, Lay::bytes, ctx->stream>>>(M, O, pat, 1, pl);
        GBS_CUDA(ctx, cudaGetLastError());
        st = gbs_timing_end(ctx);
        if (st) return st;
        zbins_chunk_kernel<<<(unsigned)nch, 64, 0, ctx->stream>>>(nb, pl.partials, pl.unit_off + 1, chunks);
        zbins_final_kernel<<<1, 64, 0, ctx->stream>>>(M, nch, chunks, logdet, pl.pflags, pl.overflow,
                                                       G + (size_t)2 * nb * j, bad);
        GBS_CUDA(ctx, cudaGetLastError());
    }
    if (even && jmax < h)
        mirror_kernel<<<(unsigned)(h - jmax), 64, 0, ctx->stream>>>(nb, h, jmax, G);
    const long long tot = (long long)(K + 1) * nb;
    sector_dft_kernel<<<(unsigned)((tot + 127) / 128), 128, 0, ctx->stream>>>(M, L, rho, K, G, bad, pkn);
    GBS_CUDA(ctx, cudaGetLastError());
    return GBS_OK;
}
}  // namespace

int sector_distribution(gbs_ctx *ctx, int M, const double *O, const double *logdet, int L, double rho, int K,
                        int even, int precision, double *pkn) {
    if (precision == GBS_FF) return sector_distribution_in<zf>(ctx, M, O, logdet, L, rho, K, even, pkn);
    if (precision == GBS_FP64) return sector_distribution_in<zc>(ctx, M, O, logdet, L, rho, K, even, pkn);
    return gbs_fail(ctx, GBS_E_INVALID, "gbs_sector_distribution: precision %d (GBS_FP64 or GBS_FF)", precision);
}
