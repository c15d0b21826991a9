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

// signed product: the unsigned product minus 2^128 (b [a < 0] + a [b < 0]), bits 112..239
__device__ __forceinline__ fx operator*(const fx &a, const fx &b) {
    uint32_t p3, p4, p5, p6, p7;
    fx_mul_upper(a, b, p3, p4, p5, p6, p7);
    const uint32_t ma = (uint32_t)((int32_t)a.w[3] >> 31), mb = (uint32_t)((int32_t)b.w[3] >> 31);
    asm("sub.cc.u32 %0, %0, %4;\n\t"
        "subc.cc.u32 %1, %1, %5;\n\t"
        "subc.cc.u32 %2, %2, %6;\n\t"
        "subc.u32 %3, %3, %7;"
        : "+r"(p4), "+r"(p5), "+r"(p6), "+r"(p7)
        : "r"(b.w[0] & ma), "r"(b.w[1] & ma), "r"(b.w[2] & ma), "r"(b.w[3] & ma));
    asm("sub.cc.u32 %0, %0, %4;\n\t"
        "subc.cc.u32 %1, %1, %5;\n\t"
        "subc.cc.u32 %2, %2, %6;\n\t"
        "subc.u32 %3, %3, %7;"
        : "+r"(p4), "+r"(p5), "+r"(p6), "+r"(p7)
        : "r"(a.w[0] & mb), "r"(a.w[1] & mb), "r"(a.w[2] & mb), "r"(a.w[3] & mb));
    fx r;
    r.w[0] = __funnelshift_r(p3, p4, 16);
    r.w[1] = __funnelshift_r(p4, p5, 16);
    r.w[2] = __funnelshift_r(p5, p6, 16);
    r.w[3] = __funnelshift_r(p6, p7, 16);
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

// det^{-1/2} for det in [2^-8, 4]: double estimate y, one Newton step y (1 + e/2),
// e = 1 - det y^2, in fixed point: relative error ~ (3/8) (2^-52)^2.
__device__ __forceinline__ fx fx_rsqrt(const fx &det) {
    const double y = rsqrt(fx_to_double(det));
    const fx y0 = fx_from_double(y);
    const fx e = fx_one() - det * (y0 * y0);
    return y0 + fx_half(y0 * e);
}
