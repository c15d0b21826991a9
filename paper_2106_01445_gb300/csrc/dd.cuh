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
// 1/sqrt(x): double estimate, then one Newton step y + y (1 - x y^2) / 2 in dd
__device__ __forceinline__ dd dd_rsqrt(dd x) {
    double y = rsqrt(x.hi);
    dd yy = dd(y);
    dd r = dd(1.0) - x * (yy * yy);
    return yy + yy * r * dd(0.5);
}
