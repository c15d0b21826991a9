// 128-bit signed fixed point on the integer pipes: value = X * 2^-112 (Q16.112),
// X two's complement in four 32-bit limbs (w[0] least significant).
//
// Used for the Schur updates of the exact sweep, whose entries are bounded: A = I - O
// = sigma_Q^{-1} <= 2 I, so every Schur complement of A has entries in [-2, 2]; with
// pivot determinants >= 2^-8 (checked, see fx_pivot_bad) the inverse pivots, the rows
// W = B P^{-1} and every intermediate of c - w0 b0 - w1 b1 stay below 2^15.  Products
// are truncated to 2^-112 (partial products below bit 96 are dropped, error < 2^-13
// of the last place); sums are exact.
#pragma once
#include <stdint.h>

#include "dd.cuh"

struct fx {
    uint32_t w[4];
};

__device__ __forceinline__ fx fx_zero() { return fx{{0u, 0u, 0u, 0u}}; }
__device__ __forceinline__ fx fx_one() { return fx{{0u, 0u, 0u, 1u << 16}}; }

__device__ __forceinline__ fx operator+(const fx &a, const fx &b) {
    fx r;
    asm("add.cc.u32 %0, %4, %8;\n\t"
        "addc.cc.u32 %1, %5, %9;\n\t"
        "addc.cc.u32 %2, %6, %10;\n\t"
        "addc.u32 %3, %7, %11;"
        : "=r"(r.w[0]), "=r"(r.w[1]), "=r"(r.w[2]), "=r"(r.w[3])
        : "r"(a.w[0]), "r"(a.w[1]), "r"(a.w[2]), "r"(a.w[3]), "r"(b.w[0]), "r"(b.w[1]), "r"(b.w[2]),
          "r"(b.w[3]));
    return r;
}
__device__ __forceinline__ fx operator-(const fx &a, const fx &b) {
    fx r;
    asm("sub.cc.u32 %0, %4, %8;\n\t"
        "subc.cc.u32 %1, %5, %9;\n\t"
        "subc.cc.u32 %2, %6, %10;\n\t"
        "subc.u32 %3, %7, %11;"
        : "=r"(r.w[0]), "=r"(r.w[1]), "=r"(r.w[2]), "=r"(r.w[3])
        : "r"(a.w[0]), "r"(a.w[1]), "r"(a.w[2]), "r"(a.w[3]), "r"(b.w[0]), "r"(b.w[1]), "r"(b.w[2]),
          "r"(b.w[3]));
    return r;
}
__device__ __forceinline__ fx operator-(const fx &a) { return fx_zero() - a; }
__device__ __forceinline__ fx &operator+=(fx &a, const fx &b) { return a = a + b; }
__device__ __forceinline__ bool fx_positive(const fx &a) {
    return (int32_t)a.w[3] > 0 || (a.w[3] == 0u && (a.w[2] | a.w[1] | a.w[0]) != 0u);
}
__device__ __forceinline__ bool operator>(const fx &a, const fx &b) { return fx_positive(a - b); }

// Limbs 3..7 of the unsigned 256-bit product a*b, without the partial products of
// columns 0 and 1 and the low halves of column 2.  Row i adds a_i * b; after row i
// the partial sum is below 2^(32 (i + 5)), so each row's carry ends in its last limb.
__device__ __forceinline__ void fx_mul_upper(const fx &a, const fx &b, uint32_t &p3, uint32_t &p4,
                                             uint32_t &p5, uint32_t &p6, uint32_t &p7) {
    // row 0: lo(a0 b3) -> 3; hi(a0 b2) -> 3, hi(a0 b3) -> 4
    asm("mul.lo.u32 %0, %2, %3;\n\t"
        "mad.hi.cc.u32 %0, %2, %4, %0;\n\t"
        "madc.hi.u32 %1, %2, %3, 0;"
        : "=&r"(p3), "=&r"(p4)
        : "r"(a.w[0]), "r"(b.w[3]), "r"(b.w[2]));
    // row 1: lo(a1 b2) -> 3, lo(a1 b3) -> 4, carry -> 5; hi(a1 b1) -> 3, hi(a1 b2) -> 4, hi(a1 b3) -> 5
    asm("mad.lo.cc.u32 %0, %3, %5, %0;\n\t"
        "madc.lo.cc.u32 %1, %3, %6, %1;\n\t"
        "addc.u32 %2, 0, 0;\n\t"
        "mad.hi.cc.u32 %0, %3, %4, %0;\n\t"
        "madc.hi.cc.u32 %1, %3, %5, %1;\n\t"
        "madc.hi.u32 %2, %3, %6, %2;"
        : "+r"(p3), "+r"(p4), "=&r"(p5)
        : "r"(a.w[1]), "r"(b.w[1]), "r"(b.w[2]), "r"(b.w[3]));
    // row 2: lo(a2 b1..b3) -> 3..5, carry -> 6; hi(a2 b0..b3) -> 3..6
    asm("mad.lo.cc.u32 %0, %4, %6, %0;\n\t"
        "madc.lo.cc.u32 %1, %4, %7, %1;\n\t"
        "madc.lo.cc.u32 %2, %4, %8, %2;\n\t"
        "addc.u32 %3, 0, 0;\n\t"
        "mad.hi.cc.u32 %0, %4, %5, %0;\n\t"
        "madc.hi.cc.u32 %1, %4, %6, %1;\n\t"
        "madc.hi.cc.u32 %2, %4, %7, %2;\n\t"
        "madc.hi.u32 %3, %4, %8, %3;"
        : "+r"(p3), "+r"(p4), "+r"(p5), "=&r"(p6)
        : "r"(a.w[2]), "r"(b.w[0]), "r"(b.w[1]), "r"(b.w[2]), "r"(b.w[3]));
    // row 3: lo(a3 b0..b3) -> 3..6, carry -> 7; hi(a3 b0..b3) -> 4..7
    asm("mad.lo.cc.u32 %0, %5, %6, %0;\n\t"
        "madc.lo.cc.u32 %1, %5, %7, %1;\n\t"
        "madc.lo.cc.u32 %2, %5, %8, %2;\n\t"
        "madc.lo.cc.u32 %3, %5, %9, %3;\n\t"
        "addc.u32 %4, 0, 0;\n\t"
        "mad.hi.cc.u32 %1, %5, %6, %1;\n\t"
        "madc.hi.cc.u32 %2, %5, %7, %2;\n\t"
        "madc.hi.cc.u32 %3, %5, %8, %3;\n\t"
        "madc.hi.u32 %4, %5, %9, %4;"
        : "+r"(p3), "+r"(p4), "+r"(p5), "+r"(p6), "=&r"(p7)
        : "r"(a.w[3]), "r"(b.w[0]), "r"(b.w[1]), "r"(b.w[2]), "r"(b.w[3]));
}

// bits 112..239 of the product held in limbs 3..7
__device__ __forceinline__ fx fx_shift_out(uint32_t p3, uint32_t p4, uint32_t p5, uint32_t p6, uint32_t p7) {
    fx r;
    r.w[0] = __funnelshift_r(p3, p4, 16);
    r.w[1] = __funnelshift_r(p4, p5, 16);
    r.w[2] = __funnelshift_r(p5, p6, 16);
    r.w[3] = __funnelshift_r(p6, p7, 16);
    return r;
}
// p4..p7 -= m & x  (the two's-complement correction 2^128 x [sign] of a signed factor)
__device__ __forceinline__ void fx_sub_masked(uint32_t &p4, uint32_t &p5, uint32_t &p6, uint32_t &p7,
                                              const fx &x, uint32_t m) {
    asm("sub.cc.u32 %0, %0, %4;\n\t"
        "subc.cc.u32 %1, %1, %5;\n\t"
        "subc.cc.u32 %2, %2, %6;\n\t"
        "subc.u32 %3, %3, %7;"
        : "+r"(p4), "+r"(p5), "+r"(p6), "+r"(p7)
        : "r"(x.w[0] & m), "r"(x.w[1] & m), "r"(x.w[2] & m), "r"(x.w[3] & m));
}
__device__ __forceinline__ uint32_t fx_sign_mask(const fx &a) { return (uint32_t)((int32_t)a.w[3] >> 31); }

// signed product: the unsigned product minus 2^128 (b [a < 0] + a [b < 0]), bits 112..239
__device__ __forceinline__ fx operator*(const fx &a, const fx &b) {
    uint32_t p3, p4, p5, p6, p7;
    fx_mul_upper(a, b, p3, p4, p5, p6, p7);
    fx_sub_masked(p4, p5, p6, p7, b, fx_sign_mask(a));
    fx_sub_masked(p4, p5, p6, p7, a, fx_sign_mask(b));
    return fx_shift_out(p3, p4, p5, p6, p7);
}
// a * b for a, b >= 0
__device__ __forceinline__ fx fx_mul_uu(const fx &a, const fx &b) {
    uint32_t p3, p4, p5, p6, p7;
    fx_mul_upper(a, b, p3, p4, p5, p6, p7);
    return fx_shift_out(p3, p4, p5, p6, p7);
}
// a * b for b >= 0, a of either sign
__device__ __forceinline__ fx fx_mul_su(const fx &a, const fx &b) {
    uint32_t p3, p4, p5, p6, p7;
    fx_mul_upper(a, b, p3, p4, p5, p6, p7);
    fx_sub_masked(p4, p5, p6, p7, b, fx_sign_mask(a));
    return fx_shift_out(p3, p4, p5, p6, p7);
}
__device__ __forceinline__ fx fx_abs(const fx &a) {
    const uint32_t m = fx_sign_mask(a);
    fx x;
#pragma unroll
    for (int k = 0; k < 4; ++k) x.w[k] = a.w[k] ^ m;
    fx r;
    asm("sub.cc.u32 %0, %4, %8;\n\t"
        "subc.cc.u32 %1, %5, %8;\n\t"
        "subc.cc.u32 %2, %6, %8;\n\t"
        "subc.u32 %3, %7, %8;"
        : "=r"(r.w[0]), "=r"(r.w[1]), "=r"(r.w[2]), "=r"(r.w[3])
        : "r"(x.w[0]), "r"(x.w[1]), "r"(x.w[2]), "r"(x.w[3]), "r"(m));
    return r;
}
// a + k 2^-16 for a small integer k (top limb only: no carry below)
__device__ __forceinline__ fx fx_add_top(const fx &a, int k) {
    fx r = a;
    r.w[3] = (uint32_t)((int32_t)a.w[3] + k);
    return r;
}
__device__ __forceinline__ fx &operator*=(fx &a, const fx &b) { return a = a * b; }
// a / 2 (arithmetic shift)
__device__ __forceinline__ fx fx_half(const fx &a) {
    fx r;
    r.w[0] = __funnelshift_r(a.w[0], a.w[1], 1);
    r.w[1] = __funnelshift_r(a.w[1], a.w[2], 1);
    r.w[2] = __funnelshift_r(a.w[2], a.w[3], 1);
    r.w[3] = (uint32_t)((int32_t)a.w[3] >> 1);
    return r;
}

__device__ __forceinline__ fx fx_from_i128(__int128 v) {
    fx r;
    r.w[0] = (uint32_t)v;
    r.w[1] = (uint32_t)(v >> 32);
    r.w[2] = (uint32_t)(v >> 64);
    r.w[3] = (uint32_t)(v >> 96);
    return r;
}
__device__ __forceinline__ __int128 fx_to_i128(const fx &a) {
    const unsigned __int128 u = (unsigned __int128)a.w[0] | ((unsigned __int128)a.w[1] << 32) |
                                ((unsigned __int128)a.w[2] << 64) | ((unsigned __int128)a.w[3] << 96);
    return (__int128)u;
}
// exact for |d| < 2^15 down to 2^-112 (lower bits truncated toward zero); zero outside
__device__ __forceinline__ fx fx_from_double(double d) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(d);
    const int ex = (int)((bits >> 52) & 0x7ff);
    if (ex == 0) return fx_zero();
    const unsigned long long mant = (bits & ((1ull << 52) - 1)) | (1ull << 52);
    const int s = ex - 963;  // d * 2^112 = mant * 2^(ex - 1075 + 112)
    if (s > 74) return fx_zero();  // |d| >= 2^15 (or not finite): outside the format
    unsigned __int128 v;
    if (s >= 0) v = (unsigned __int128)mant << s;
    else v = s > -64 ? (unsigned __int128)(mant >> (-s)) : (unsigned __int128)0;
    __int128 x = (__int128)v;
    if (bits >> 63) x = -x;
    return fx_from_i128(x);
}
// nearest-double leading part of a
__device__ __forceinline__ double fx_to_double(const fx &a) {
    const long long hi = (long long)(((unsigned long long)a.w[3] << 32) | a.w[2]);
    return (double)hi * 0x1p-48;
}
// a as a double-double (the top 64 bits rounded to a double, the remainder below)
__device__ __forceinline__ dd fx_to_dd(const fx &a) {
    const long long hi = (long long)(((unsigned long long)a.w[3] << 32) | a.w[2]);
    const unsigned long long lo = ((unsigned long long)a.w[1] << 32) | a.w[0];
    const double h = (double)hi;
    const long long rem = hi - (long long)h;  // |rem| <= 2^10: exact
    const double l = (double)rem + (double)lo * 0x1p-64;
    const dd s = dd_quick_two_sum(h, l);
    return dd(s.hi * 0x1p-48, s.lo * 0x1p-48);
}

// pivot check: 0 fine, 1 not positive, 2 below the fixed-point range (det < 2^-8)
__device__ __forceinline__ int fx_pivot_bad(const fx &det) {
    if (!fx_positive(det)) return 1;
    return (int32_t)det.w[3] < 256 ? 2 : 0;
}
// the same for a pivot block given by p00 and det: both positive, det >= 2^-8
__device__ __forceinline__ int fx_chol_bad(const fx &p00, const fx &det) {
    if (!fx_positive(p00)) return 1;
    return fx_pivot_bad(det);
}

// floor(A R / 2^64) for A < 2^127 and R < 2^64 (limbs of columns 2..5 of the 192-bit
// product); the partial products of columns 0 and 1 are dropped (result low by <= 3)
__device__ __forceinline__ fx fx_mul_r64(const fx &a, unsigned long long R) {
    const uint32_t r0 = (uint32_t)R, r1 = (uint32_t)(R >> 32);
    fx q;
    asm("mul.lo.u32 %0, %6, %8;\n\t"
        "mul.lo.u32 %1, %7, %8;\n\t"
        "mad.hi.cc.u32 %0, %5, %8, %0;\n\t"
        "madc.hi.cc.u32 %1, %6, %8, %1;\n\t"
        "madc.hi.u32 %2, %7, %8, 0;\n\t"
        "mad.lo.cc.u32 %0, %5, %9, %0;\n\t"
        "madc.lo.cc.u32 %1, %6, %9, %1;\n\t"
        "madc.lo.cc.u32 %2, %7, %9, %2;\n\t"
        "addc.u32 %3, 0, 0;\n\t"
        "mad.hi.cc.u32 %0, %4, %9, %0;\n\t"
        "madc.hi.cc.u32 %1, %5, %9, %1;\n\t"
        "madc.hi.cc.u32 %2, %6, %9, %2;\n\t"
        "madc.hi.u32 %3, %7, %9, %3;"
        : "=&r"(q.w[0]), "=&r"(q.w[1]), "=&r"(q.w[2]), "=&r"(q.w[3])
        : "r"(a.w[0]), "r"(a.w[1]), "r"(a.w[2]), "r"(a.w[3]), "r"(r0), "r"(r1));
    return q;
}

// x^{-1/2} for x in [2^-16, 2^16) (pivots lie in [2^-8, 4]), built for a short
// dependency chain (Newton's iteration r <- r + r e / 2, e = 1 - x r^2):
//  * x = x_m 4^h with x_m = W / 2^64 in [1/4, 1), W the 64 bits after the leading zeros;
//  * an FP32 estimate of r = x_m^{-1/2} in (1, 2] (~22 bits);
//  * two Newton steps on W in 64-bit integer arithmetic, R = r 2^61 (~56 bits);
//  * one Newton step against the whole of x: e from the top 128 bits of X R^2 (X the
//    normalised 128-bit x), then y += y e / 2 (error ~ (3/2) e^2 + truncation 2^-110).
// Inputs outside the range (checked by the callers) give a finite, meaningless result.
static __device__ __noinline__ fx fx_rsqrt(fx x) {
    uint32_t lz = __clz(x.w[3]);
    lz = lz < 1u ? 1u : (lz > 31u ? 31u : lz);
    int k = 16 - (int)lz;  // x = (W / 2^64) 2^k
    unsigned long long W = ((unsigned long long)__funnelshift_l(x.w[2], x.w[3], lz) << 32) |
                           __funnelshift_l(x.w[1], x.w[2], lz);
    const int odd = k & 1;
    W >>= odd;
    k += odd;
    const int h = k / 2;
    // FP32 estimate, turned into R = r 2^61 through its bits
    const float rf = rsqrtf(__uint2float_rn((uint32_t)(W >> 32)) * 0x1p-32f);
    const uint32_t fb = __float_as_uint(rf);
    int s0 = (int)((fb >> 23) & 0xffu) - 127 + 38;
    s0 = s0 < 0 ? 0 : (s0 > 39 ? 39 : s0);
    unsigned long long R = (unsigned long long)((fb & 0x7fffffu) | 0x800000u) << s0;
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const unsigned long long S = __umul64hi(R, R);         // r^2 2^58
        const unsigned long long P = __umul64hi(W, S);         // x_m r^2 2^58
        const long long E = (long long)((1ull << 58) - P);     // e 2^58
        R += (unsigned long long)__mul64hi((long long)R, (long long)((unsigned long long)E << 5));
    }
    // y = r 2^-h in Q16.112: Y = R 2^(51 - h)
    int s2 = 19 - h;
    s2 = s2 < 11 ? 11 : (s2 > 26 ? 26 : s2);
    const uint32_t q0 = (uint32_t)R, q1 = (uint32_t)(R >> 32);
    const fx y{{0u, q0 << s2, __funnelshift_l(q0, q1, s2), q1 >> (32 - s2)}};
    // e = 1 - x y^2 = 1 - T2 2^(-121 - odd), T2 = top 128 bits of X_n R^2, X_n = X 2^(lz - 1)
    const int sx = (int)lz - 1;
    const fx xn{{x.w[0] << sx, __funnelshift_l(x.w[0], x.w[1], sx), __funnelshift_l(x.w[1], x.w[2], sx),
                 __funnelshift_l(x.w[2], x.w[3], sx)}};
    const fx t2 = fx_mul_r64(fx_mul_r64(xn, R), R);
    const int se = 9 + odd;  // e in units of 2^-112: its low 64 bits suffice (|e| < 2^-50)
    const unsigned long long tl = ((unsigned long long)__funnelshift_r(t2.w[1], t2.w[2], se) << 32) |
                                  __funnelshift_r(t2.w[0], t2.w[1], se);
    const long long E = -(long long)tl;
    // y e / 2 in units of 2^-112: R E 2^(-62 - h)
    const unsigned long long plo = R * (unsigned long long)E;
    const long long phi = __mul64hi((long long)R, E);
    int sd = 62 + h;
    sd = sd < 55 ? 55 : (sd > 70 ? 70 : sd);
    const long long dlt = sd < 64 ? (long long)(((unsigned long long)phi << (64 - sd)) | (plo >> sd))
                                  : (phi >> (sd - 64));
    const uint32_t ext = (uint32_t)(dlt >> 63);
    return y + fx{{(uint32_t)dlt, (uint32_t)((unsigned long long)dlt >> 32), ext, ext}};
}
// det of the SPD 2x2 block [[p00, p01], [p01, p11]]
__device__ __forceinline__ fx fx_det2(const fx &p00, const fx &p01, const fx &p11) {
    const fx a = fx_abs(p01);
    return fx_mul_uu(p00, p11) - fx_mul_uu(a, a);
}

// Symmetric form of the 2x2 block elimination used by the fixed-point sweep.  With
// the pivot block P = R R^T (R lower triangular, 1/r00 = a, r10, 1/r11 = b), the
// Schur update C - B P^{-1} B^T equals C - U U^T, U = B R^{-T}: row i of U is
// u0 = b_i0 a, u1 = (b_i1 - r10 u0) b = b_i1 b - u0 c with c = r10 b = p01 det^{-1/2}
// (two products side by side).  |u_ik| <= sqrt(c_ii) <= sqrt(2), so the rows
// are stored offset, u' = u + 2 > 0, and each entry needs two unsigned products:
//   c_ij - u_i . u_j = c_ij - (u'_i0 u'_j0 + u'_i1 u'_j1) + t_i + t_j,  t = 2 (u'0 + u'1) - 4.
struct fx_piv {
    fx a, c, b, rs, det;
};
// the Cholesky quantities from a = p00^{-1/2} and rs = det^{-1/2} (independent, so the
// two rsqrts need not wait for each other): b = x^{-1/2} = rs sqrt(p00) = rs p00 a
__device__ __forceinline__ fx_piv fx_pivot_from(const fx &p00, const fx &p01, const fx &det, const fx &a,
                                               const fx &rs) {
    fx_piv v;
    v.a = a;
    v.rs = rs;
    v.det = det;
    v.c = fx_mul_su(p01, rs);
    v.b = fx_mul_uu(rs, fx_mul_uu(p00, a));
    return v;
}
__device__ __forceinline__ fx_piv fx_pivot(const fx &p00, const fx &p01, const fx &p11) {
    const fx det = fx_det2(p00, p01, p11);
    return fx_pivot_from(p00, p01, det, fx_rsqrt(p00), fx_rsqrt(det));
}
// offset row (u'0, u'1, t) of U from the pivot-row entries b0 = P(0, .), b1 = P(1, .)
__device__ __forceinline__ void fx_urow(const fx_piv &v, const fx &b0, const fx &b1, fx &u0, fx &u1, fx &t) {
    const fx x0 = fx_mul_su(b0, v.a);
    const fx x1 = fx_mul_su(b1, v.b) - x0 * v.c;
    u0 = fx_add_top(x0, 2 << 16);
    u1 = fx_add_top(x1, 2 << 16);
    const fx s = u0 + u1;
    t = fx_add_top(s + s, -(4 << 16));
}
// c - u_i . u_j from the offset rows
__device__ __forceinline__ fx fx_sym_update(const fx &c, const fx &ui0, const fx &ui1, const fx &ti,
                                            const fx &uj0, const fx &uj1, const fx &tj) {
    return ((c + ti) + tj) - (fx_mul_uu(ui0, uj0) + fx_mul_uu(ui1, uj1));
}

// ---- prefactors as mantissa x 2^e, and exponent-aligned sums -------------------------
// The breadth-first prefactors (products of up to seven det^{-1/2} in [1/2, 16]) leave
// the fixed-point range, so they are kept as m 2^e with m in [1, 2).
struct __align__(16) fxe {
    fx m;
    int e;
};
__device__ __forceinline__ fxe fxe_one() { return fxe{fx_one(), 0}; }
// a >> k for 0 <= k <= 31 (arithmetic)
__device__ __forceinline__ fx fx_shr_small(const fx &a, int k) {
    fx r;
    r.w[0] = __funnelshift_r(a.w[0], a.w[1], k);
    r.w[1] = __funnelshift_r(a.w[1], a.w[2], k);
    r.w[2] = __funnelshift_r(a.w[2], a.w[3], k);
    r.w[3] = (uint32_t)((int32_t)a.w[3] >> k);
    return r;
}
// a << k for 0 <= k <= 31
__device__ __forceinline__ fx fx_shl_small(const fx &a, int k) {
    fx r;
    r.w[3] = __funnelshift_l(a.w[2], a.w[3], k);
    r.w[2] = __funnelshift_l(a.w[1], a.w[2], k);
    r.w[1] = __funnelshift_l(a.w[0], a.w[1], k);
    r.w[0] = a.w[0] << k;
    return r;
}
// a >> s for any s >= 0 (arithmetic; s >= 127 leaves the sign)
__device__ __forceinline__ fx fx_shr(const fx &a, int s) {
    const uint32_t sg = (uint32_t)((int32_t)a.w[3] >> 31);
    if (s > 127) s = 127;
    const int q = s >> 5, b = s & 31;
    // limb shift by q (selects, no indexed local memory), then the bit shift
    const uint32_t w0 = q == 0 ? a.w[0] : q == 1 ? a.w[1] : q == 2 ? a.w[2] : a.w[3];
    const uint32_t w1 = q == 0 ? a.w[1] : q == 1 ? a.w[2] : q == 2 ? a.w[3] : sg;
    const uint32_t w2 = q == 0 ? a.w[2] : q == 1 ? a.w[3] : sg;
    const uint32_t w3 = q == 0 ? a.w[3] : sg;
    return fx_shr_small(fx{{w0, w1, w2, w3}}, b);
}
// m r 2^e renormalised, for r in (0, 32)
__device__ __forceinline__ fxe fxe_mul(const fxe &a, const fx &r) {
    const fx p = fx_mul_uu(a.m, r);  // (0, 64)
    const int k = (31 - __clz((int)p.w[3])) - 16;  // floor(log2 p), in [-2, 5] for p >= 1/4
    fxe o;
    o.m = k >= 0 ? fx_shr_small(p, k) : fx_shl_small(p, -k);
    o.e = a.e + k;
    return o;
}
// m 2^e as a double-double
__device__ __forceinline__ dd fxe_to_dd(const fxe &a) {
    const dd v = fx_to_dd(a.m);
    const double s = ldexp(1.0, a.e);
    return dd(v.hi * s, v.lo * s);
}
__device__ __forceinline__ fx fx_shfl_xor(const fx &a, int mask) {
    fx r;
#pragma unroll
    for (int k = 0; k < 4; ++k) r.w[k] = __shfl_xor_sync(0xffffffffu, a.w[k], mask);
    return r;
}
__device__ __forceinline__ fx fx_neg_if(const fx &a, bool neg) { return neg ? -a : a; }
