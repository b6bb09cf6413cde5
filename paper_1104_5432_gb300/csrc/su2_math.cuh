// su2_math.cuh -- the transcendental pieces of the heat-bath draw.
//
// FP64 takes ln u and sin/cos(2 pi u) of its uniforms from tables and short
// series (ln_u01_tab, sincospi_tab, at the end of this file; each checked
// on every grid point against CUDA's log and sincospi by su2_selftest_ln /
// su2_selftest_trig), and CUDA's accurate sqrt and rsqrt (the reciprocal
// square root within 1 ulp, instead of a division by sqrt).  FP32 uses
// short forms whose
// error is bounded well inside the FP32 parity budget (2e-5 per link):
//   ln u       for u on the uniform grid ((k + 1/2) 2^-23):
//              u > 15/16: ln(1 - v) = -(v + v^2/2 + ... + v^8/8) with
//              v = 1 - u exact (Sterbenz); truncation < v^9/9 < 2e-12 v;
//              otherwise the hardware base-2 logarithm (__log2f, absolute
//              error <= 2^-22 on [1/2, 2], 2 ulp elsewhere) times ln 2,
//              i.e. relative error <= 2.6e-6 since |ln u| >= 0.0645 there.
//   cos^2(2 pi r), sin/cos(2 pi r): the hardware sine/cosine at
//              x = 2 pi (r - 1/2) in (-pi, pi), where its absolute error is
//              <= 2^-21.41; cos(2 pi r) = -cos x, sin(2 pi r) = -sin x.
//   sqrt(x), 1/sqrt(x): x rsqrtf(x), rsqrtf(x) (2 ulp).
// Both are checked exhaustively on the GPU against CUDA's accurate logf,
// cospif and sincospif over all 2^23 grid points (su2_selftest_math).
#pragma once
#include <cuda_runtime.h>

#include "su2_device.cuh"

namespace su2 {

template <typename T> struct Math;

template <> struct Math<float> {
    static __device__ __forceinline__ float ln_u01(float u)
    {
        const float v = add_(1.0f, neg_(u));
        float s = fma_(v, 0.125f, 0.142857142857f);
        s = fma_(v, s, 0.166666666667f);
        s = fma_(v, s, 0.2f);
        s = fma_(v, s, 0.25f);
        s = fma_(v, s, 0.333333333333f);
        s = fma_(v, s, 0.5f);
        s = fma_(v, s, 1.0f);
        const float near1 = mul_(neg_(v), s);
        const float far = mul_(__log2f(u), 0.693147180559945f);
        return u > 0.9375f ? near1 : far;
    }
    static __device__ __forceinline__ float cos2pi_sq(float r)
    {
        const float c = __cosf(mul_(6.28318530717959f, add_(r, -0.5f)));
        return mul_(c, c);
    }
    static __device__ __forceinline__ void sincos2pi(float r, float* s, float* c)
    {
        float sx, cx;
        __sincosf(mul_(6.28318530717959f, add_(r, -0.5f)), &sx, &cx);
        *s = -sx;
        *c = -cx;
    }
    static __device__ __forceinline__ float sqrt_pos(float x) { return mul_(x, rsqrtf(x)); }
    static __device__ __forceinline__ float log1p(float x) { return log1pf(x); }
    static __device__ __forceinline__ float expm1(float x) { return expm1f(x); }
    static __device__ __forceinline__ float rsqrt(float x) { return rsqrtf(x); }
};

// Two FP32 lanes at once: the polynomial and the scalings as packed
// operations, the hardware logarithm, cosine and reciprocal square root per
// lane; every lane gets exactly the bits Math<float> gives it.
template <> struct Math<float2> {
    static __device__ __forceinline__ float2 ln_u01(float2 u)
    {
        const float2 v = add_(splat<float2>(1.0f), neg_(u));
        float2 s = fma_(v, splat<float2>(0.125f), splat<float2>(0.142857142857f));
        s = fma_(v, s, splat<float2>(0.166666666667f));
        s = fma_(v, s, splat<float2>(0.2f));
        s = fma_(v, s, splat<float2>(0.25f));
        s = fma_(v, s, splat<float2>(0.333333333333f));
        s = fma_(v, s, splat<float2>(0.5f));
        s = fma_(v, s, splat<float2>(1.0f));
        const float2 near1 = mul_(neg_(v), s);
        const float2 far = mul_(make_float2(__log2f(u.x), __log2f(u.y)),
                                splat<float2>(0.693147180559945f));
        return make_float2(u.x > 0.9375f ? near1.x : far.x, u.y > 0.9375f ? near1.y : far.y);
    }
    static __device__ __forceinline__ float2 cos2pi_sq(float2 r)
    {
        const float2 x = mul_(splat<float2>(6.28318530717959f), add_(r, splat<float2>(-0.5f)));
        const float2 c = make_float2(__cosf(x.x), __cosf(x.y));
        return mul_(c, c);
    }
    static __device__ __forceinline__ void sincos2pi(float2 r, float2* s, float2* c)
    {
        const float2 x = mul_(splat<float2>(6.28318530717959f), add_(r, splat<float2>(-0.5f)));
        float sx, cx, sy, cy;
        __sincosf(x.x, &sx, &cx);
        __sincosf(x.y, &sy, &cy);
        *s = make_float2(-sx, -sy);
        *c = make_float2(-cx, -cy);
    }
    static __device__ __forceinline__ float2 sqrt_pos(float2 x)
    {
        return mul_(x, make_float2(rsqrtf(x.x), rsqrtf(x.y)));
    }
    static __device__ __forceinline__ float2 rsqrt(float2 x)
    {
        return make_float2(rsqrtf(x.x), rsqrtf(x.y));
    }
};

template <> struct Math<double> {
    static __device__ __forceinline__ double ln_u01(double u) { return log(u); }
    static __device__ __forceinline__ double cos2pi_sq(double r)
    {
        const double c = cospi(mul_(2.0, r));
        return mul_(c, c);
    }
    // (the FP64 kernels take these from sincospi_tab; kept for the generic
    // forms)
    static __device__ __forceinline__ void sincos2pi(double r, double* s, double* c)
    {
        const double x = mul_(2.0, r);
        *c = cospi(x);
        *s = cospi(add_(x, -0.5));
    }
    static __device__ __forceinline__ double sqrt_pos(double x) { return sqrt(x); }
    static __device__ __forceinline__ double log1p(double x) { return ::log1p(x); }
    static __device__ __forceinline__ double expm1(double x) { return ::expm1(x); }
    static __device__ __forceinline__ double rsqrt(double x) { return ::rsqrt(x); }
};

// ln u for the FP64 path's uniform u = (2 (w >> 9) + 1) 2^-24, table-driven
// after Tang (ACM TOMS 15 (1989) 144): u = 2^n m with m in [0.75, 1.5) read
// off the bits, c the centre of m's table interval, g = 1/c rounded and
// -ln g stored (computed once on the host in extended precision),
// r = m g - 1 with one fused multiply-add (|r| <= 2^-9 / 0.75; the
// interval just below 1 takes c = 1, r = m - 1 exactly), and
//   ln u = n ln 2 - ln g + ln(1 + r),
//   ln(1 + r) = r + r^2 (-1/2 + r (1/3 + r (-1/4 + r (1/5 - r/6))))
// (the Taylor series; the first term left out is below r^7/7 < 2e-19).
// ln 2 = hi + lo with hi's low mantissa bits zero, so that n hi is exact.
// Ten FP64 instructions against ~30 instruction times for a general log:
// on GB300 the FP64 unit is the heat bath's bottleneck in FP64.
// The FP64 tables (fill_fp64_table): the logarithm's 256 intervals, ln 2
// as (hi, lo), then (cos, sin) of pi j / 128, j = 0 .. 255.
constexpr int TAB_LN = 0, TAB_LN2 = 256, TAB_TRIG = 257, FP64_TABLE_ENTRIES = 513;

__device__ __forceinline__ double ln_u01_tab(uint32_t w, const double2* __restrict__ tab)
{
    const uint32_t a = 2u * (w >> 9) + 1u;  // u = a 2^-24, 1 <= a < 2^24
    const int p = 31 - __clz((int)a);     // 2^p <= a < 2^(p+1)
    // the first 8 fraction bits of M = a 2^-p in [1, 2): the table interval
    const uint32_t t = (p >= 8 ? a >> (p - 8) : a << (8 - p)) & 255u;
    const int h = t >= 128 ? 1 : 0;         // M >= 1.5: m = M / 2
    const int n = p - 24 + h;
    const double m = exact_double((int32_t)a, -p - h);
    const double2 e = __ldg(tab + TAB_LN + t);  // (g, -ln g)
    const double2 l2 = __ldg(tab + TAB_LN2);    // (ln 2 hi, ln 2 lo)
    const double r = fma_(m, e.x, -1.0);
    double q = fma_(r, -1.0 / 6.0, 0.2);
    q = fma_(r, q, -0.25);
    q = fma_(r, q, 1.0 / 3.0);
    q = fma_(r, q, -0.5);
    const double lp = fma_(mul_(r, r), q, r);
    const double nd = n ? exact_double(n, 0) : 0.0;
    return add_(fma_(nd, l2.x, e.y), fma_(nd, l2.y, lp));
}

// sin(pi y) and cos(pi y) for y = num 2^-bits in [0, 2] (num <= 2^(bits+1),
// bits >= 8), table-driven: y = j / 128 + d with j the nearest multiple
// (read off the bits) and |d| <= 1/256, b = pi d, and from the table's
// (cos, sin) of pi j / 128 = (C, S):
//   cos(pi y) = C + (C (cos b - 1) - S sin b),
//   sin(pi y) = S + (S (cos b - 1) + C sin b),
// with cos b - 1 = b^2 (-1/2 + b^2 (1/24 - b^2 / 720)) and
// sin b = b + b^3 (-1/6 + b^2 (1/120 - b^2 / 5040)), the Taylor series
// (|b| <= pi/256: the first terms left out are below 1e-19).  Fifteen FP64
// instructions for both, thirteen for the cosine alone, against ~15
// instruction times for one general cospi.
__device__ __forceinline__ void sincospi_tab(uint32_t num, int bits,
                                             const double2* __restrict__ tab, double* sn,
                                             double* cs)
{
    const int sh = bits - 7;
    const uint32_t j = (num + (1u << (sh - 1))) >> sh;  // nearest j / 128
    const int32_t res = (int32_t)num - (int32_t)(j << sh);  // d = res 2^-bits
    const double2 t = __ldg(tab + TAB_TRIG + (j & 255u));  // (C, S)
    // b = pi d: res 2^-bits exact, one rounding for the product with pi
    const double b = res ? mul_(exact_double(res, -bits), 3.141592653589793) : 0.0;
    const double b2 = mul_(b, b);
    const double cm1 = mul_(b2, fma_(b2, fma_(b2, -1.0 / 720.0, 1.0 / 24.0), -0.5));
    const double sb = fma_(mul_(b, b2), fma_(b2, fma_(b2, -1.0 / 5040.0, 1.0 / 120.0), -1.0 / 6.0), b);
    *cs = add_(t.x, fma_(t.x, cm1, neg_(mul_(t.y, sb))));
    *sn = add_(t.y, fma_(t.y, cm1, mul_(t.x, sb)));
}

}  // namespace su2
