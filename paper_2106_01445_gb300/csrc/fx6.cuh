// 192-bit signed fixed point (Q16.176) on the integer pipes: value = X * 2^-176, X two's
// complement in six 32-bit limbs (w[0] least significant).  The same representation,
// bounds and truncated products as the 128-bit fx (fx.cuh), 64 bits wider: per-term
// relative error ~2^-164 instead of ~2^-100, for signed sums that cancel by kappa up to
// ~1e30 (the 30-click anchors of the 100-mode workload cancel by ~1e27).  Prefactors and
// sums are carried as m 2^e with the 192-bit mantissa (fxe6), never in double-double.
#pragma once
#include <stdint.h>

#include "fx.cuh"

struct fx6 {
    uint32_t w[6];
};

__device__ __forceinline__ fx6 fx6_zero() { return fx6{{0u, 0u, 0u, 0u, 0u, 0u}}; }
__device__ __forceinline__ fx6 fx6_one() { return fx6{{0u, 0u, 0u, 0u, 0u, 1u << 16}}; }

__device__ __forceinline__ fx6 operator+(const fx6 &a, const fx6 &b) {
    fx6 r;
    asm("add.cc.u32 %0, %6, %12;\n\t"
        "addc.cc.u32 %1, %7, %13;\n\t"
        "addc.cc.u32 %2, %8, %14;\n\t"
        "addc.cc.u32 %3, %9, %15;\n\t"
        "addc.cc.u32 %4, %10, %16;\n\t"
        "addc.u32 %5, %11, %17;"
        : "=r"(r.w[0]), "=r"(r.w[1]), "=r"(r.w[2]), "=r"(r.w[3]), "=r"(r.w[4]), "=r"(r.w[5])
        : "r"(a.w[0]), "r"(a.w[1]), "r"(a.w[2]), "r"(a.w[3]), "r"(a.w[4]), "r"(a.w[5]), "r"(b.w[0]),
          "r"(b.w[1]), "r"(b.w[2]), "r"(b.w[3]), "r"(b.w[4]), "r"(b.w[5]));
    return r;
}
__device__ __forceinline__ fx6 operator-(const fx6 &a, const fx6 &b) {
    fx6 r;
    asm("sub.cc.u32 %0, %6, %12;\n\t"
        "subc.cc.u32 %1, %7, %13;\n\t"
        "subc.cc.u32 %2, %8, %14;\n\t"
        "subc.cc.u32 %3, %9, %15;\n\t"
        "subc.cc.u32 %4, %10, %16;\n\t"
        "subc.u32 %5, %11, %17;"
        : "=r"(r.w[0]), "=r"(r.w[1]), "=r"(r.w[2]), "=r"(r.w[3]), "=r"(r.w[4]), "=r"(r.w[5])
        : "r"(a.w[0]), "r"(a.w[1]), "r"(a.w[2]), "r"(a.w[3]), "r"(a.w[4]), "r"(a.w[5]), "r"(b.w[0]),
          "r"(b.w[1]), "r"(b.w[2]), "r"(b.w[3]), "r"(b.w[4]), "r"(b.w[5]));
    return r;
}
__device__ __forceinline__ fx6 operator-(const fx6 &a) { return fx6_zero() - a; }
__device__ __forceinline__ fx6 &operator+=(fx6 &a, const fx6 &b) { return a = a + b; }
__device__ __forceinline__ bool fx_positive(const fx6 &a) {
    return (int32_t)a.w[5] > 0 || (a.w[5] == 0u && (a.w[4] | a.w[3] | a.w[2] | a.w[1] | a.w[0]) != 0u);
}
__device__ __forceinline__ bool operator>(const fx6 &a, const fx6 &b) { return fx_positive(a - b); }
__device__ __forceinline__ uint32_t fx_sign_mask(const fx6 &a) { return (uint32_t)((int32_t)a.w[5] >> 31); }

// Limbs 5..11 of the unsigned 384-bit product a*b, without the partial products of
// columns 0..3 and the low halves of column 4 (the carry they would send into column 5
// is lost: the result below is low by a few 2^-16 of its last place).  Row i adds a_i * b;
// after row i the partial sum is below 2^(32 (i + 7)), so each row's carry ends in its
// last limb.
__device__ __forceinline__ void fx6_mul_upper(const fx6 &a, const fx6 &b, uint32_t &p5, uint32_t &p6, uint32_t &p7,
                                              uint32_t &p8, uint32_t &p9, uint32_t &p10, uint32_t &p11) {
    // row 0
    asm("mul.lo.u32 %0, %2, %8;\n\t"
        "mad.hi.cc.u32 %0, %2, %7, %0;\n\t"
        "madc.hi.u32 %1, %2, %8, 0;"
        : "=&r"(p5), "=&r"(p6)
        : "r"(a.w[0]), "r"(b.w[0]), "r"(b.w[1]), "r"(b.w[2]), "r"(b.w[3]), "r"(b.w[4]), "r"(b.w[5]));
    // row 1
    asm("mad.lo.cc.u32 %0, %3, %8, %0;\n\t"
        "madc.lo.cc.u32 %1, %3, %9, %1;\n\t"
        "addc.u32 %2, 0, 0;\n\t"
        "mad.hi.cc.u32 %0, %3, %7, %0;\n\t"
        "madc.hi.cc.u32 %1, %3, %8, %1;\n\t"
        "madc.hi.u32 %2, %3, %9, %2;"
        : "+r"(p5), "+r"(p6), "=&r"(p7)
        : "r"(a.w[1]), "r"(b.w[0]), "r"(b.w[1]), "r"(b.w[2]), "r"(b.w[3]), "r"(b.w[4]), "r"(b.w[5]));
    // row 2
    asm("mad.lo.cc.u32 %0, %4, %8, %0;\n\t"
        "madc.lo.cc.u32 %1, %4, %9, %1;\n\t"
        "madc.lo.cc.u32 %2, %4, %10, %2;\n\t"
        "addc.u32 %3, 0, 0;\n\t"
        "mad.hi.cc.u32 %0, %4, %7, %0;\n\t"
        "madc.hi.cc.u32 %1, %4, %8, %1;\n\t"
        "madc.hi.cc.u32 %2, %4, %9, %2;\n\t"
        "madc.hi.u32 %3, %4, %10, %3;"
        : "+r"(p5), "+r"(p6), "+r"(p7), "=&r"(p8)
        : "r"(a.w[2]), "r"(b.w[0]), "r"(b.w[1]), "r"(b.w[2]), "r"(b.w[3]), "r"(b.w[4]), "r"(b.w[5]));
    // row 3
    asm("mad.lo.cc.u32 %0, %5, %8, %0;\n\t"
        "madc.lo.cc.u32 %1, %5, %9, %1;\n\t"
        "madc.lo.cc.u32 %2, %5, %10, %2;\n\t"
        "madc.lo.cc.u32 %3, %5, %11, %3;\n\t"
        "addc.u32 %4, 0, 0;\n\t"
        "mad.hi.cc.u32 %0, %5, %7, %0;\n\t"
        "madc.hi.cc.u32 %1, %5, %8, %1;\n\t"
        "madc.hi.cc.u32 %2, %5, %9, %2;\n\t"
        "madc.hi.cc.u32 %3, %5, %10, %3;\n\t"
        "madc.hi.u32 %4, %5, %11, %4;"
        : "+r"(p5), "+r"(p6), "+r"(p7), "+r"(p8), "=&r"(p9)
        : "r"(a.w[3]), "r"(b.w[0]), "r"(b.w[1]), "r"(b.w[2]), "r"(b.w[3]), "r"(b.w[4]), "r"(b.w[5]));
    // row 4
    asm("mad.lo.cc.u32 %0, %6, %8, %0;\n\t"
        "madc.lo.cc.u32 %1, %6, %9, %1;\n\t"
        "madc.lo.cc.u32 %2, %6, %10, %2;\n\t"
        "madc.lo.cc.u32 %3, %6, %11, %3;\n\t"
        "madc.lo.cc.u32 %4, %6, %12, %4;\n\t"
        "addc.u32 %5, 0, 0;\n\t"
        "mad.hi.cc.u32 %0, %6, %7, %0;\n\t"
        "madc.hi.cc.u32 %1, %6, %8, %1;\n\t"
        "madc.hi.cc.u32 %2, %6, %9, %2;\n\t"
        "madc.hi.cc.u32 %3, %6, %10, %3;\n\t"
        "madc.hi.cc.u32 %4, %6, %11, %4;\n\t"
        "madc.hi.u32 %5, %6, %12, %5;"
        : "+r"(p5), "+r"(p6), "+r"(p7), "+r"(p8), "+r"(p9), "=&r"(p10)
        : "r"(a.w[4]), "r"(b.w[0]), "r"(b.w[1]), "r"(b.w[2]), "r"(b.w[3]), "r"(b.w[4]), "r"(b.w[5]));
    // row 5
    asm("mad.lo.cc.u32 %0, %7, %8, %0;\n\t"
        "madc.lo.cc.u32 %1, %7, %9, %1;\n\t"
        "madc.lo.cc.u32 %2, %7, %10, %2;\n\t"
        "madc.lo.cc.u32 %3, %7, %11, %3;\n\t"
        "madc.lo.cc.u32 %4, %7, %12, %4;\n\t"
        "madc.lo.cc.u32 %5, %7, %13, %5;\n\t"
        "addc.u32 %6, 0, 0;\n\t"
        "mad.hi.cc.u32 %1, %7, %8, %1;\n\t"
        "madc.hi.cc.u32 %2, %7, %9, %2;\n\t"
        "madc.hi.cc.u32 %3, %7, %10, %3;\n\t"
        "madc.hi.cc.u32 %4, %7, %11, %4;\n\t"
        "madc.hi.cc.u32 %5, %7, %12, %5;\n\t"
        "madc.hi.u32 %6, %7, %13, %6;"
        : "+r"(p5), "+r"(p6), "+r"(p7), "+r"(p8), "+r"(p9), "+r"(p10), "=&r"(p11)
        : "r"(a.w[5]), "r"(b.w[0]), "r"(b.w[1]), "r"(b.w[2]), "r"(b.w[3]), "r"(b.w[4]), "r"(b.w[5]));
}
// bits 176..367 of the product held in limbs 5..11
__device__ __forceinline__ fx6 fx6_shift_out(uint32_t p5, uint32_t p6, uint32_t p7, uint32_t p8, uint32_t p9,
                                             uint32_t p10, uint32_t p11) {
    fx6 r;
    r.w[0] = __funnelshift_r(p5, p6, 16);
    r.w[1] = __funnelshift_r(p6, p7, 16);
    r.w[2] = __funnelshift_r(p7, p8, 16);
    r.w[3] = __funnelshift_r(p8, p9, 16);
    r.w[4] = __funnelshift_r(p9, p10, 16);
    r.w[5] = __funnelshift_r(p10, p11, 16);
    return r;
}
// p6..p11 -= m & x  (the two's-complement correction 2^192 x [sign] of a signed factor)
__device__ __forceinline__ void fx6_sub_masked(uint32_t &p6, uint32_t &p7, uint32_t &p8, uint32_t &p9,
                                               uint32_t &p10, uint32_t &p11, const fx6 &x, uint32_t m) {
    asm("sub.cc.u32 %0, %0, %6;\n\t"
        "subc.cc.u32 %1, %1, %7;\n\t"
        "subc.cc.u32 %2, %2, %8;\n\t"
        "subc.cc.u32 %3, %3, %9;\n\t"
        "subc.cc.u32 %4, %4, %10;\n\t"
        "subc.u32 %5, %5, %11;"
        : "+r"(p6), "+r"(p7), "+r"(p8), "+r"(p9), "+r"(p10), "+r"(p11)
        : "r"(x.w[0] & m), "r"(x.w[1] & m), "r"(x.w[2] & m), "r"(x.w[3] & m), "r"(x.w[4] & m), "r"(x.w[5] & m));
}
// signed product: the unsigned product minus 2^192 (b [a < 0] + a [b < 0]), bits 176..367
__device__ __forceinline__ fx6 operator*(const fx6 &a, const fx6 &b) {
    uint32_t p5, p6, p7, p8, p9, p10, p11;
    fx6_mul_upper(a, b, p5, p6, p7, p8, p9, p10, p11);
    fx6_sub_masked(p6, p7, p8, p9, p10, p11, b, fx_sign_mask(a));
    fx6_sub_masked(p6, p7, p8, p9, p10, p11, a, fx_sign_mask(b));
    return fx6_shift_out(p5, p6, p7, p8, p9, p10, p11);
}
__device__ __forceinline__ fx6 fx_mul_uu(const fx6 &a, const fx6 &b) {  // a, b >= 0
    uint32_t p5, p6, p7, p8, p9, p10, p11;
    fx6_mul_upper(a, b, p5, p6, p7, p8, p9, p10, p11);
    return fx6_shift_out(p5, p6, p7, p8, p9, p10, p11);
}
__device__ __forceinline__ fx6 fx_mul_su(const fx6 &a, const fx6 &b) {  // b >= 0
    uint32_t p5, p6, p7, p8, p9, p10, p11;
    fx6_mul_upper(a, b, p5, p6, p7, p8, p9, p10, p11);
    fx6_sub_masked(p6, p7, p8, p9, p10, p11, b, fx_sign_mask(a));
    return fx6_shift_out(p5, p6, p7, p8, p9, p10, p11);
}
__device__ __forceinline__ fx6 fx_abs(const fx6 &a) { return fx_sign_mask(a) ? -a : a; }
// a + k 2^-16 for a small integer k (top limb only)
__device__ __forceinline__ fx6 fx_add_top(const fx6 &a, int k) {
    fx6 r = a;
    r.w[5] = (uint32_t)((int32_t)a.w[5] + k);
    return r;
}
// d * 2^176 as a 192-bit integer: exact for 2^-123 <= |d| < 2^15 (all 53 bits of d lie
// above 2^-176), truncated toward zero below; zero outside the format
__device__ __forceinline__ fx6 fx6_from_double(double d) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(d);
    const int ex = (int)((bits >> 52) & 0x7ff);
    if (ex == 0) return fx6_zero();
    unsigned long long mant = (bits & ((1ull << 52) - 1)) | (1ull << 52);
    int s = ex - 899;  // d * 2^176 = mant * 2^(ex - 1075 + 176)
    if (s > 138) return fx6_zero();  // |d| >= 2^15 (or not finite)
    if (s < 0) {
        if (s <= -53) return fx6_zero();
        mant >>= -s;
        s = 0;
    }
    const int q = s >> 5, b = s & 31;
    const uint32_t m0 = (uint32_t)mant, m1 = (uint32_t)(mant >> 32);
    const uint32_t l0 = m0 << b, l1 = __funnelshift_l(m0, m1, b), l2 = b ? (m1 >> (32 - b)) : 0u;
    fx6 r;
#pragma unroll
    for (int i = 0; i < 6; ++i) r.w[i] = i == q ? l0 : (i == q + 1 ? l1 : (i == q + 2 ? l2 : 0u));
    return (bits >> 63) ? -r : r;
}
// the leading 128 bits as the 4-limb fx (truncated toward minus infinity)
__device__ __forceinline__ fx fx6_top(const fx6 &a) { return fx{{a.w[2], a.w[3], a.w[4], a.w[5]}}; }
__device__ __forceinline__ fx6 fx6_widen(const fx &a) { return fx6{{0u, 0u, a.w[0], a.w[1], a.w[2], a.w[3]}}; }
__device__ __forceinline__ double fx_to_double(const fx6 &a) { return fx_to_double(fx6_top(a)); }
__device__ __forceinline__ int fx_pivot_bad(const fx6 &det) {
    if (!fx_positive(det)) return 1;
    return (int32_t)det.w[5] < 256 ? 2 : 0;
}
__device__ __forceinline__ int fx_chol_bad(const fx6 &p00, const fx6 &det) {
    if (!fx_positive(p00)) return 1;
    return fx_pivot_bad(det);
}
// x^{-1/2}: the 128-bit reciprocal square root of x's leading 128 bits (relative error
// ~2^-104 for x >= 2^-8), then one Newton step in 192 bits, y <- y + y e / 2 with
// e = 1 - x y^2 (error ~ (3/2) e^2 + truncation ~2^-170)
static __device__ __noinline__ fx6 fx6_rsqrt(fx6 x) {
    const fx6 y = fx6_widen(fx_rsqrt(fx6_top(x)));
    const fx6 e = fx6_one() - fx_mul_uu(x, fx_mul_uu(y, y));
    const fx6 d = fx_mul_su(e, y);
    fx6 h;  // d / 2 (arithmetic shift)
#pragma unroll
    for (int k = 0; k < 5; ++k) h.w[k] = __funnelshift_r(d.w[k], d.w[k + 1], 1);
    h.w[5] = (uint32_t)((int32_t)d.w[5] >> 1);
    return y + h;
}
__device__ __forceinline__ fx6 fx_det2(const fx6 &p00, const fx6 &p01, const fx6 &p11) {
    const fx6 a = fx_abs(p01);
    return fx_mul_uu(p00, p11) - fx_mul_uu(a, a);
}

// the symmetric 2x2 block elimination of the fixed-point sweep (see fx_piv in fx.cuh)
struct fx6_piv {
    fx6 a, c, b, rs, det;
};
__device__ __forceinline__ fx6_piv fx_pivot_from(const fx6 &p00, const fx6 &p01, const fx6 &det, const fx6 &a,
                                                const fx6 &rs) {
    fx6_piv v;
    v.a = a;
    v.rs = rs;
    v.det = det;
    v.c = fx_mul_su(p01, rs);
    v.b = fx_mul_uu(rs, fx_mul_uu(p00, a));
    return v;
}
__device__ __forceinline__ fx6_piv fx_pivot(const fx6 &p00, const fx6 &p01, const fx6 &p11) {
    const fx6 det = fx_det2(p00, p01, p11);
    return fx_pivot_from(p00, p01, det, fx6_rsqrt(p00), fx6_rsqrt(det));
}
__device__ __forceinline__ void fx_urow(const fx6_piv &v, const fx6 &b0, const fx6 &b1, fx6 &u0, fx6 &u1, fx6 &t) {
    const fx6 x0 = fx_mul_su(b0, v.a);
    const fx6 x1 = fx_mul_su(b1, v.b) - x0 * v.c;
    u0 = fx_add_top(x0, 2 << 16);
    u1 = fx_add_top(x1, 2 << 16);
    const fx6 s = u0 + u1;
    t = fx_add_top(s + s, -(4 << 16));
}
__device__ __forceinline__ fx6 fx_sym_update(const fx6 &c, const fx6 &ui0, const fx6 &ui1, const fx6 &ti,
                                             const fx6 &uj0, const fx6 &uj1, const fx6 &tj) {
    return ((c + ti) + tj) - (fx_mul_uu(ui0, uj0) + fx_mul_uu(ui1, uj1));
}

// ---- m 2^e with a 192-bit mantissa: prefactors, sub-unit and unit sums --------------------
// m is kept with |m| in [1, 2) (or zero); products renormalise, sums align to the larger
// exponent (the smaller addend loses its bits below 2^-176 of the larger).
struct fxe6 {
    fx6 m;
    int e;
    fxe6() = default;
    __device__ fxe6(const fx6 &mm, int ee) : m(mm), e(ee) {}
    __device__ explicit fxe6(double v) : m(fx6_from_double(v)), e(0) {}  // v in [1, 2) or 0 (1.0 here)
};
__device__ __forceinline__ fx6 fx_shr_small(const fx6 &a, int k) {  // 0 <= k <= 31, arithmetic
    fx6 r;
#pragma unroll
    for (int i = 0; i < 5; ++i) r.w[i] = __funnelshift_r(a.w[i], a.w[i + 1], k);
    r.w[5] = (uint32_t)((int32_t)a.w[5] >> k);
    return r;
}
__device__ __forceinline__ fx6 fx_shl_small(const fx6 &a, int k) {  // 0 <= k <= 31
    fx6 r;
#pragma unroll
    for (int i = 5; i > 0; --i) r.w[i] = __funnelshift_l(a.w[i - 1], a.w[i], k);
    r.w[0] = a.w[0] << k;
    return r;
}
// a >> s for any s >= 0 (arithmetic; s >= 191 leaves the sign)
__device__ __forceinline__ fx6 fx_shr(const fx6 &a, int s) {
    const uint32_t sg = fx_sign_mask(a);
    if (s > 191) s = 191;
    const int q = s >> 5, b = s & 31;
    fx6 t;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        uint32_t v = sg;
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (k == i + q) v = a.w[k];
        t.w[i] = v;
    }
    return fx_shr_small(t, b);
}
// floor(log2 |m|) relative to 1 (m != 0), from the leading limbs
__device__ __forceinline__ int fx6_log2(const fx6 &m) {
    const fx6 a = fx_abs(m);
#pragma unroll
    for (int i = 5; i >= 0; --i)
        if (a.w[i]) return (31 - __clz((int)a.w[i])) + 32 * i - 176;
    return -100000;
}
__device__ __forceinline__ fxe6 fxe6_norm(const fx6 &m, int e) {
    const int k = fx6_log2(m);
    if (k < -176) return fxe6(fx6_zero(), -(1 << 20));
    fx6 r = m;
    int kk = k;
    while (kk > 0) { const int s = kk > 31 ? 31 : kk; r = fx_shr_small(r, s); kk -= s; }
    while (kk < 0) { const int s = -kk > 31 ? 31 : -kk; r = fx_shl_small(r, s); kk += s; }
    return fxe6(r, e + k);
}
__device__ __forceinline__ fxe6 operator*(const fxe6 &a, const fxe6 &b) {
    if (!fx_positive(fx_abs(a.m)) || !fx_positive(fx_abs(b.m))) return fxe6(fx6_zero(), -(1 << 20));
    return fxe6_norm(a.m * b.m, a.e + b.e);
}
__device__ __forceinline__ fxe6 fxe6_add(const fxe6 &a, const fxe6 &b) {
    const bool az = !fx_positive(fx_abs(a.m)), bz = !fx_positive(fx_abs(b.m));
    if (az) return b;
    if (bz) return a;
    const fxe6 &hi = a.e >= b.e ? a : b, &lo = a.e >= b.e ? b : a;
    return fxe6_norm(hi.m + fx_shr(lo.m, hi.e - lo.e), hi.e);
}
// a prefactor r in (0, 32) as m 2^e
__device__ __forceinline__ fxe6 fxe6_from(const fx6 &r) { return fxe6_norm(r, 0); }
__device__ __forceinline__ fxe6 fxe_mul(const fxe6 &a, const fx6 &r) { return a * fxe6_from(r); }
__device__ __forceinline__ double fxe6_to_double(const fxe6 &a) { return ldexp(fx_to_double(a.m), a.e); }
__device__ __forceinline__ fx6 fx_shfl_xor(const fx6 &a, int mask) {
    fx6 r;
#pragma unroll
    for (int k = 0; k < 6; ++k) r.w[k] = __shfl_xor_sync(0xffffffffu, a.w[k], mask);
    return r;
}
__device__ __forceinline__ fx6 fx_neg_if(const fx6 &a, bool neg) { return neg ? -a : a; }
