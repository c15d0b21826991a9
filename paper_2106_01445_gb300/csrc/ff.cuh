// Float-float arithmetic on the FP32 pipes (Dekker 1971; the FMA forms of Hida, Li &
// Bailey 2001): a value is hi + lo with |lo| <= ulp(hi)/2, ~48 significant bits.  On
// a GPU whose FP64 rate is 1/64 of FP32 this carries FP64-class precision at a
// fraction of FP64's cost.  Additions are the "sloppy" form (error ~2^-46 of the
// operands' magnitude), products use FMA for the exact low part of hi*hi.
#pragma once

struct ff {
    float hi, lo;
    ff() = default;
    __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
    // nearest float plus the remainder: exact to ~2^-48 relative
    __host__ __device__ ff(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
};

__device__ __forceinline__ ff ff_quick_two_sum(float s, float e) {
    const float h = s + e;
    return ff(h, e - (h - s));
}
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
    const float s = a + b, bp = s - a;
    return ff(s, (a - (s - bp)) + (b - bp));
}
__device__ __forceinline__ ff operator+(ff a, ff b) {
    const ff s = ff_two_sum(a.hi, b.hi);
    return ff_quick_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__device__ __forceinline__ ff operator*(ff a, ff b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    return ff_quick_two_sum(p, e);
}
// a / b: quotient of the high parts, one correction from the remainder
__device__ __forceinline__ ff operator/(ff a, ff b) {
    const float q1 = a.hi / b.hi;
    const ff r = a - b * ff(q1, 0.0f);
    return ff_quick_two_sum(q1, r.hi / b.hi);
}
__device__ __forceinline__ bool operator>(ff a, ff b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
// 1/sqrt(x): float estimate y, one Newton step y (1 + r/2), r = 1 - x y^2
__device__ __forceinline__ ff ff_rsqrt(ff x) {
    const float y = rsqrtf(x.hi);
    const float p = y * y, ep = fmaf(y, y, -p);
    const ff r = ff(1.0f, 0.0f) - x * ff(p, ep);
    return ff_quick_two_sum(y, 0.5f * y * r.hi);
}
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// Fused forms for complex products (FMA error-free products of the high parts, the sum of
// the high parts by TwoSum, every low-order term in one FMA chain, one renormalisation):
// x0 y0 + x1 y1 in 19 FP32 operations and e - x0 y0 - x1 y1 in 27, against 46 and 68 for
// the same through separate products and sums; error ~2^-46 of the terms' magnitudes.
__device__ __forceinline__ ff ff_dot2(ff x0, ff y0, ff x1, ff y1) {
    const float p0 = x0.hi * y0.hi, q0 = fmaf(x0.hi, y0.hi, -p0);
    const float p1 = x1.hi * y1.hi, q1 = fmaf(x1.hi, y1.hi, -p1);
    const ff s = ff_two_sum(p0, p1);
    float lo = s.lo + (q0 + q1);
    lo = fmaf(x0.hi, y0.lo, lo);
    lo = fmaf(x0.lo, y0.hi, lo);
    lo = fmaf(x1.hi, y1.lo, lo);
    lo = fmaf(x1.lo, y1.hi, lo);
    return ff_quick_two_sum(s.hi, lo);
}
__device__ __forceinline__ ff ff_fms2(ff e, ff x0, ff y0, ff x1, ff y1) {
    const float p0 = x0.hi * y0.hi, q0 = fmaf(x0.hi, y0.hi, -p0);
    const float p1 = x1.hi * y1.hi, q1 = fmaf(x1.hi, y1.hi, -p1);
    const ff s1 = ff_two_sum(e.hi, -p0);
    const ff s2 = ff_two_sum(s1.hi, -p1);
    float lo = e.lo + (s1.lo + s2.lo) - (q0 + q1);
    lo = fmaf(-x0.hi, y0.lo, lo);
    lo = fmaf(-x0.lo, y0.hi, lo);
    lo = fmaf(-x1.hi, y1.lo, lo);
    lo = fmaf(-x1.lo, y1.hi, lo);
    return ff_quick_two_sum(s2.hi, lo);
}
