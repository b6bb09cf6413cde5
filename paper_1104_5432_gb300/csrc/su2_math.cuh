// su2_math.cuh -- the transcendental pieces of the heat-bath draw.
//
// FP64 uses CUDA's accurate double functions (the reciprocal square root
// through rsqrt, within 1 ulp, instead of a division by sqrt).  FP32 uses
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

namespace su2 {

template <typename T> struct Math;

template <> struct Math<float> {
    static __device__ __forceinline__ float ln_u01(float u)
    {
        const float v = 1.0f - u;
        float s = fmaf(v, 0.125f, 0.142857142857f);
        s = fmaf(v, s, 0.166666666667f);
        s = fmaf(v, s, 0.2f);
        s = fmaf(v, s, 0.25f);
        s = fmaf(v, s, 0.333333333333f);
        s = fmaf(v, s, 0.5f);
        s = fmaf(v, s, 1.0f);
        const float near1 = -v * s;
        const float far = __log2f(u) * 0.693147180559945f;
        return u > 0.9375f ? near1 : far;
    }
    static __device__ __forceinline__ float cos2pi_sq(float r)
    {
        const float c = __cosf(6.28318530717959f * (r - 0.5f));
        return c * c;
    }
    static __device__ __forceinline__ void sincos2pi(float r, float* s, float* c)
    {
        float sx, cx;
        __sincosf(6.28318530717959f * (r - 0.5f), &sx, &cx);
        *s = -sx;
        *c = -cx;
    }
    static __device__ __forceinline__ float sqrt_pos(float x) { return x * rsqrtf(x); }
    static __device__ __forceinline__ float log1p(float x) { return log1pf(x); }
    static __device__ __forceinline__ float expm1(float x) { return expm1f(x); }
    static __device__ __forceinline__ float rsqrt(float x) { return rsqrtf(x); }
};

template <> struct Math<double> {
    static __device__ __forceinline__ double ln_u01(double u) { return log(u); }
    static __device__ __forceinline__ double cos2pi_sq(double r)
    {
        const double c = cospi(2.0 * r);
        return c * c;
    }
    static __device__ __forceinline__ void sincos2pi(double r, double* s, double* c)
    {
        sincospi(2.0 * r, s, c);
    }
    static __device__ __forceinline__ double sqrt_pos(double x) { return sqrt(x); }
    static __device__ __forceinline__ double log1p(double x) { return ::log1p(x); }
    static __device__ __forceinline__ double expm1(double x) { return ::expm1(x); }
    static __device__ __forceinline__ double rsqrt(double x) { return ::rsqrt(x); }
};

}  // namespace su2
