// Complex FP64 arithmetic for the sector-resolved sweep (the generating-function
// variable t of the photon-number sectors is taken on a circle in the complex plane).
#pragma once
#include <math.h>

struct zc {
    double re, im;
    zc() = default;
    __host__ __device__ zc(double r) : re(r), im(0.0) {}
    __host__ __device__ zc(double r, double i) : re(r), im(i) {}
};

__device__ __forceinline__ zc operator+(zc a, zc b) { return zc(a.re + b.re, a.im + b.im); }
__device__ __forceinline__ zc operator-(zc a, zc b) { return zc(a.re - b.re, a.im - b.im); }
__device__ __forceinline__ zc operator-(zc a) { return zc(-a.re, -a.im); }
__device__ __forceinline__ zc operator*(zc a, zc b) {
    return zc(fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re));
}
__device__ __forceinline__ zc &operator+=(zc &a, zc b) { return a = a + b; }
__device__ __forceinline__ bool zc_nan(zc a) { return a.re != a.re || a.im != a.im; }

// principal 1/sqrt(z), z != 0: sqrt(z) = (s, y / 2s), s = sqrt((|z| + x) / 2) for x >= 0
// (the mirrored form for x < 0), then its reciprocal
__device__ __forceinline__ zc zc_rsqrt(zc z) {
    const double r = hypot(z.re, z.im);
    double sr, si;
    if (z.re >= 0.0) {
        sr = sqrt(0.5 * (r + z.re));
        si = z.im / (2.0 * sr);
    } else {
        const double s = sqrt(0.5 * (r - z.re));
        sr = fabs(z.im) / (2.0 * s);
        si = copysign(s, z.im);
    }
    const double q = 1.0 / (sr * sr + si * si);
    return zc(sr * q, -si * q);
}

// Complex float-float (~48-bit parts on the FP32 pipes): the same sweep at a fraction of
// complex FP64's cost where its precision suffices.
#include "ff.cuh"

struct zf {
    ff re, im;
    zf() = default;
    __host__ __device__ zf(double r) : re(r), im(0.0f, 0.0f) {}
    __host__ __device__ zf(ff r, ff i) : re(r), im(i) {}
};

__device__ __forceinline__ zf operator+(zf a, zf b) { return zf(a.re + b.re, a.im + b.im); }
__device__ __forceinline__ zf operator-(zf a, zf b) { return zf(a.re - b.re, a.im - b.im); }
__device__ __forceinline__ zf operator-(zf a) { return zf(-a.re, -a.im); }
__device__ __forceinline__ zf operator*(zf a, zf b) {
    return zf(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
__device__ __forceinline__ zf &operator+=(zf &a, zf b) { return a = a + b; }
__device__ __forceinline__ bool zf_nan(zf a) { return a.re.hi != a.re.hi || a.im.hi != a.im.hi; }

// principal 1/sqrt(z), z != 0, as zc_rsqrt: |z| and the half-angle root from two reciprocal
// square roots, 1/sqrt(z) = conj(sqrt z) / |z|
__device__ __forceinline__ zf zf_rsqrt(zf z) {
    const ff n2 = z.re * z.re + z.im * z.im;
    const ff ra = ff_rsqrt(n2);  // 1 / |z|
    const ff a = n2 * ra;        // |z|
    const ff half(0.5f, 0.0f);
    ff sr, si;
    if (z.re.hi >= 0.0f) {
        const ff h = (a + z.re) * half;
        const ff rh = ff_rsqrt(h);
        sr = h * rh;
        si = z.im * rh * half;
    } else {
        const ff h = (a - z.re) * half;
        const ff rh = ff_rsqrt(h);
        const ff s = h * rh;
        const ff ay = z.im.hi < 0.0f ? -z.im : z.im;
        sr = ay * rh * half;
        si = z.im.hi < 0.0f ? -s : s;
    }
    return zf(sr * ra, -(si * ra));
}
