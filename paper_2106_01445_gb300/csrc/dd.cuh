// Double-double arithmetic on the FP64 pipes (Dekker 1971; Hida, Li & Bailey,
// "Algorithms for quad-double precision floating point arithmetic", 2001).
// A value is hi + lo, |lo| <= ulp(hi)/2: ~106 significant bits.  Additions use
// the "sloppy" form (error ~2^-106 (|a| + |b|)), products use FMA for the exact
// low part of hi*hi.
#pragma once

struct dd {
    double hi, lo;
    __host__ __device__ constexpr dd() : hi(0.0), lo(0.0) {}
    __host__ __device__ constexpr dd(double h) : hi(h), lo(0.0) {}
    __host__ __device__ constexpr dd(double h, double l) : hi(h), lo(l) {}
};

__device__ __forceinline__ dd dd_quick_two_sum(double a, double b) {
    double s = a + b;
    return dd(s, b - (s - a));
}
__device__ __forceinline__ dd dd_two_sum(double a, double b) {
    double s = a + b;
    double bp = s - a;
    return dd(s, (a - (s - bp)) + (b - bp));
}
__device__ __forceinline__ dd operator+(dd a, dd b) {
    dd s = dd_two_sum(a.hi, b.hi);
    return dd_quick_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }
__device__ __forceinline__ dd operator*(dd a, dd b) {
    double p = a.hi * b.hi;
    double e = fma(a.hi, b.hi, -p);
    e = fma(a.hi, b.lo, e);
    e = fma(a.lo, b.hi, e);
    return dd_quick_two_sum(p, e);
}
__device__ __forceinline__ dd operator/(dd a, dd b) {
    double q1 = a.hi / b.hi;
    dd r = a - b * dd(q1);
    double q2 = r.hi / b.hi;
    r = r - b * dd(q2);
    double q3 = r.hi / b.hi;
    return dd_quick_two_sum(q1, q2) + dd(q3);
}
__device__ __forceinline__ dd &operator+=(dd &a, dd b) { return a = a + b; }
__device__ __forceinline__ dd &operator-=(dd &a, dd b) { return a = a - b; }
__device__ __forceinline__ dd &operator*=(dd &a, dd b) { return a = a * b; }
__device__ __forceinline__ bool operator>(dd a, dd b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ bool operator==(dd a, dd b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ dd dd_abs(dd a) { return a.hi < 0.0 ? -a : a; }
// 1/sqrt(x): double estimate y, then one Newton step y (1 + r/2), r = 1 - x y^2.
// y^2 and x.hi y^2 are split exactly with FMA; since x.hi y^2 is within a few ulps
// of 1, 1 - x.hi y^2 is exact (Sterbenz) and r is the residual to ~2^-106.  The
// neglected Newton term 3 r^2 / 8 is of order 2^-105.
__device__ __forceinline__ dd dd_rsqrt(dd x) {
    const double y = rsqrt(x.hi);
    const double p = y * y, ep = fma(y, y, -p);
    const double t = x.hi * p, et = fma(x.hi, p, -t);
    double r = (1.0 - t) - et;
    r = fma(-x.hi, ep, r);
    r = fma(-x.lo, p, r);
    return dd_quick_two_sum(y, 0.5 * y * r);
}

// Fused forms for the Schur updates: the exact products of the high parts enter
// through TwoSum, every term of order 2^-53 relative is gathered in one double,
// and the result is renormalised once.  Error ~2^-104 of the largest magnitude
// involved, as for the sloppy addition.
// a0 b0 + a1 b1
__device__ __forceinline__ dd dd_dot2(dd a0, dd b0, dd a1, dd b1) {
    const double p0 = a0.hi * b0.hi, e0 = fma(a0.hi, b0.hi, -p0);
    const double p1 = a1.hi * b1.hi, e1 = fma(a1.hi, b1.hi, -p1);
    const dd s = dd_two_sum(p0, p1);
    const double l0 = fma(a0.hi, b0.lo, fma(a0.lo, b0.hi, e0));
    const double l1 = fma(a1.hi, b1.lo, fma(a1.lo, b1.hi, e1));
    return dd_quick_two_sum(s.hi, (l0 + l1) + s.lo);
}
// c - a0 b0 - a1 b1
__device__ __forceinline__ dd dd_fms2(dd c, dd a0, dd b0, dd a1, dd b1) {
    const double p0 = a0.hi * b0.hi, e0 = fma(a0.hi, b0.hi, -p0);
    const double p1 = a1.hi * b1.hi, e1 = fma(a1.hi, b1.hi, -p1);
    const dd s = dd_two_sum(c.hi, -p0);
    const dd s2 = dd_two_sum(s.hi, -p1);
    double lo = fma(-a0.hi, b0.lo, c.lo);
    lo = fma(-a0.lo, b0.hi, lo);
    lo = fma(-a1.hi, b1.lo, lo);
    lo = fma(-a1.lo, b1.hi, lo);
    lo = (lo - (e0 + e1)) + (s.lo + s2.lo);
    return dd_quick_two_sum(s2.hi, lo);
}
